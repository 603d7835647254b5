// Correction weights for (target, triangle) pairs, one warp per pair.
//
// For a pair (x, T) the weights are (subtract-and-add, Section 3.6)
//     C_k = w_k sum_a K_a(xi_k) m_a - [k != own] W_k G(x, y_k),
//     m_a = int_T G(x, y) K_a(rho_T^{-1}(y)) dA,
// i.e. the exact integral of G against the discrete L2 projection of the
// density onto P_4 minus what the far sum already added for T's nodes.
// m_a comes from the near scheme (Section 3.3, adaptive subdivision with the
// ellipse stop test of Section 4.1) or the self scheme (Section 3.4,
// radius-arclength coordinates on three fans, generalized Gaussian rule in
// the radius, graded Gauss-Legendre panels in the arc length).
//
// Per quadrature point the kernels accumulate the moments mu_i of a basis of
// P_4 (the tensor-Legendre basis leg15 in FP64, monomials in (3x - 1, 3y - 1)
// in float-float); a constant matrix Q (generated in high precision) maps mu
// to the nodal weights: C_k = sum_i Q_ki mu_i - [k != own] W_k G.
// The node loops run in float-float (vp_f2.cuh: the near loop entirely, the
// self loop from the FP64 panel quantities on) or, with VP_NF_FP64_WEIGHTS,
// in FP64 with the table-driven vp_logd; the subdivision tree, the stop test
// and the panel construction are FP64 in both.
//
// Float-float near pairs take three routes: a classifier (one thread per
// pair) takes the stop test of the whole triangle; pairs whose triangle is a
// leaf go through a constant map of the far rule (k_weights_near_root); the
// others have their leaves listed by a depth-first subdivision (one thread
// per pair, counted, scanned, written) and evaluated 32 at a time
// (k_weights_near_deep).
#include "vp_internal.h"
#include "vp_f2.cuh"
#include "vp_ff.cuh"
#include "vp_weights.cuh"

namespace {

// ------------------------------------------------------------------ self
__global__ void __launch_bounds__(WARPS * 32) k_weights_self(WeightsArgs a, const int32_t* __restrict__ idx, int64_t n) {
    __shared__ LogSmem lt;
    load_logtab(a.tab, lt);
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (w >= n) return;
    const double ln2 = a.tab->ln2;
    const int64_t p = idx[w];
    const int T = a.ptri[p], t = a.ptgt[p];
    const double* v = a.tv + 6 * (int64_t)T;
    const double Ax = v[0], Ay = v[1];
    const double ex = v[2] - Ax, ey = v[3] - Ay, fx = v[4] - Ax, fy = v[5] - Ay;
    const double J = a.J[T];
    const double invJ = 1.0 / J;
    const double xx = a.txy[2 * t], xy = a.txy[2 * t + 1];
    // reference coordinates of the target (rho_T^-1 x)
    const double qx0 = xx - Ax, qy0 = xy - Ay;
    const double xi0 = (qx0 * fy - qy0 * fx) * invJ, eta0 = (ex * qy0 - ey * qx0) * invJ;
    const int own = own_index(a, t, T);
    const int gl = lane >> 1, jb = (lane & 1) * 4;
    const double lxg = a.tab->lx[gl], lwg = a.tab->lw[gl];
    double gr[4], gwl[4], glr[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        gr[q] = a.tab->gr[jb + q];
        gwl[q] = a.tab->gw[jb + q] * VP_INV_TWO_PI;
        glr[q] = a.tab->glogr[jb + q];
    }
    double m[VP_NB];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) m[q] = 0.0;
    int panels = 0;
    for (int e = 0; e < 3; e++) {
        const double Px = v[2 * e], Py = v[2 * e + 1];
        const double Qx = v[(2 * e + 2) % 6], Qy = v[(2 * e + 3) % 6];
        const double dx = rn_sub(Qx, Px), dy = rn_sub(Qy, Py);
        const double L = rn_sqrt(rn_add(rn_mul(dx, dx), rn_mul(dy, dy)));
        if (L == 0.0) continue;
        const double h = rn_div(fabs(rn_sub(rn_mul(dx, rn_sub(xy, Py)), rn_mul(dy, rn_sub(xx, Px)))), L);
        if (h == 0.0) continue;
        double st = rn_div(rn_add(rn_mul(dx, rn_sub(xx, Px)), rn_mul(dy, rn_sub(xy, Py))), L);
        if (st < 0.0) st = 0.0;
        if (st > L) st = L;
        const double fxp = rn_add(Px, rn_mul(rn_div(st, L), dx)), fyp = rn_add(Py, rn_mul(rn_div(st, L), dy));
        const double ddx = rn_sub(xx, fxp), ddy = rn_sub(xy, fyp);
        const double delta = rn_sqrt(rn_add(rn_mul(ddx, ddx), rn_mul(ddy, ddy)));
        const double Lst = rn_sub(L, st);
        // reference coordinates of P and of the direction of the side
        const double qpx = Px - Ax, qpy = Py - Ay;
        const double xiP = (qpx * fy - qpy * fx) * invJ, etaP = (ex * qpy - ey * qpx) * invJ;
        const double dxi = (dx * fy - dy * fx) * invJ, deta = (ex * dy - ey * dx) * invJ;
        for (int side = 0; side < 2; side++) {
            double len = side == 0 ? st : Lst;
            if (!(len > 0.0)) continue;
            const int Nd = dyadic_count(len, delta);
            // panel boundaries: b_0 = end, b_i = end -/+ (1 - 2^-i) len, b_{Nd+1} = st
            double b0 = side == 0 ? 0.0 : L;
            for (int i = 0; i <= Nd; i++) {
                double b1;
                if (i == Nd) b1 = st;
                else {
                    double frac = rn_mul(rn_sub(1.0, ldexp(1.0, -(i + 1))), len);
                    b1 = side == 0 ? frac : rn_sub(L, frac);
                }
                panels++;
                const double s = b0 + (b1 - b0) * lxg;
                const double ws = fabs((b1 - b0) * lwg) * h;
                const double sl = s / L;
                const double rx = Px + sl * dx - xx, ry = Py + sl * dy - xy;
                const double lr0 = 0.5 * vp_logd(rx * rx + ry * ry, lt.rc, lt.lc, ln2);
                // reference coordinates along the ray x + r (gamma(s) - x)
                const double xig = xiP + sl * dxi - xi0, etag = etaP + sl * deta - eta0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const double g = (lr0 + glr[q]) * ws * gwl[q];
                    accumulate(m, g, fma(gr[q], xig, xi0), fma(gr[q], etag, eta0));
                }
                b0 = b1;
            }
        }
    }
    finish_pair(a, p, T, own, xx, xy, m, lane, lt.rc, lt.lc, ln2);
    if (lane == 0) {
        a.pstat[p] = panels;
        a.pcap[p] = 0;
    }
}

// ------------------------------------------------------------------ near
// FP64 reference: node loop in FP64 with the table-driven vp_logd.
__global__ void __launch_bounds__(WARPS * 32) k_weights_near(WeightsArgs a, const int32_t* __restrict__ idx, int64_t n) {
    __shared__ SubTri stack_all[WARPS][STK];
    __shared__ LeafMap leaf_all[WARPS][LEAFCAP];
    __shared__ LogSmem lt;
    load_logtab(a.tab, lt);
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * WARPS + wl;
    if (w >= n) return;
    const double ln2 = a.tab->ln2;
    SubTri* stack = stack_all[wl];
    LeafMap* leaves = leaf_all[wl];
    const int64_t p = idx[w];
    const int T = a.ptri[p], t = a.ptgt[p];
    const double* v = a.tv + 6 * (int64_t)T;
    const double Ax = v[0], Ay = v[1];
    const double ex = rn_sub(v[2], Ax), ey = rn_sub(v[3], Ay), fx = rn_sub(v[4], Ax), fy = rn_sub(v[5], Ay);
    const double J = a.J[T];
    const double xx = a.txy[2 * t], xy = a.txy[2 * t + 1];
    const int own = own_index(a, t, T);
    const int Nn = a.tab->near_degree;
    const double R_root = ellipse_R_rn(a.tab->near_what, J, a.eps, a.c_near);
    const double* nx = a.tab->nx;
    const double* ny = a.tab->ny;
    const double* nw = a.tab->nw;

    double m[VP_NB];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) m[q] = 0.0;
    if (lane == 0) {
        SubTri r;
        r.v[0] = 0; r.v[1] = 0; r.v[2] = 1; r.v[3] = 0; r.v[4] = 0; r.v[5] = 1; r.L = 0;
        stack[0] = r;
    }
    __syncwarp();
    int sp = 1, nleaf = 0, total_leaves = 0, capped = 0;
    int visited = 0;              // sub-triangles examined; bounded so no input can loop for long
    bool overflow = false;
    const unsigned lower = (1u << lane) - 1u;
    while (sp > 0 || nleaf > 0) {
        bool flush = nleaf > 0 && (sp == 0 || nleaf + 32 > LEAFCAP || nleaf >= 32);
        if (!flush) {
            int c = min(sp, 32);
            c = min(c, (STK - sp) / 3);
            if (c <= 0 || visited > MAX_VISITED) {
                overflow = true;
                break;
            }
            visited += c;
            SubTri S;
            bool stop = false;
            if (lane < c) {
                S = stack[sp - 1 - lane];
                double ph[6];
                sub_phys(S, Ax, Ay, ex, ey, fx, fy, ph);
                // R_S = w J_S / (eps C) = R_T 4^-depth exactly (power-of-two scaling)
                stop = !tri_near_fast(ph, xx, xy, Nn, ldexp(R_root, -2 * S.L)) && !tri_contains_rn(ph, xx, xy);
                if (!stop && S.L >= a.depth_cap) {
                    stop = true;
                    capped++;
                }
            }
            __syncwarp();
            const unsigned lm = __ballot_sync(0xffffffffu, lane < c && stop);
            const unsigned sm = __ballot_sync(0xffffffffu, lane < c && !stop);
            sp -= c;
            if (lane < c) {
                if (stop) {
                    const double sc = ldexp(1.0, -S.L);
                    LeafMap lf;
                    lf.a0x = S.v[0] * sc;
                    lf.a0y = S.v[1] * sc;
                    lf.e1x = (S.v[2] - S.v[0]) * sc;
                    lf.e1y = (S.v[3] - S.v[1]) * sc;
                    lf.e2x = (S.v[4] - S.v[0]) * sc;
                    lf.e2y = (S.v[5] - S.v[1]) * sc;
                    lf.wJ = ldexp(J, -2 * S.L) * (0.5 * VP_INV_TWO_PI);
                    leaves[nleaf + __popc(lm & lower)] = lf;
                } else {
                    push_children(S, stack, sp + 4 * __popc(sm & lower));
                }
            }
            nleaf += __popc(lm);
            sp += 4 * __popc(sm);
            __syncwarp();
        } else {
            // near rule on every buffered leaf: (leaf, node) pairs over the lanes
            const int combos = nleaf * VP_NNEAR;
            for (int i = lane; i < combos; i += 32) {
                const int li = i / VP_NNEAR, j = i - li * VP_NNEAR;
                const LeafMap& lf = leaves[li];
                const double zx = nx[j], zy = ny[j];
                const double xi = fma(zy, lf.e2x, fma(zx, lf.e1x, lf.a0x));
                const double eta = fma(zy, lf.e2y, fma(zx, lf.e1y, lf.a0y));
                const double dx = xx - fma(eta, fx, fma(xi, ex, Ax)), dy = xy - fma(eta, fy, fma(xi, ey, Ay));
                const double g = vp_logd(dx * dx + dy * dy, lt.rc, lt.lc, ln2) * (nw[j] * lf.wJ);
                accumulate(m, g, xi, eta);
            }
            total_leaves += nleaf;
            nleaf = 0;
            __syncwarp();
        }
    }
    if (overflow && lane == 0) atomicOr(a.flag, VP_DEV_ERR_STACK);
    finish_pair(a, p, T, own, xx, xy, m, lane, lt.rc, lt.lc, ln2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) capped += __shfl_xor_sync(0xffffffffu, capped, o);
    if (lane == 0) {
        a.pstat[p] = total_leaves;
        a.pcap[p] = capped;
    }
}

// ---------------------------------------------------- near, float-float
// Leaf of the float-float node loop: node j of the near rule sits at
// reference coordinates a0 + sh z_j and at y - x = D0 + sh E_j, with
// E_j = z_j,x (B - A) + z_j,y (C - A) and sh = +-2^-L (every child of a split
// keeps its parent's orientation except the fourth, its point reflection).
struct LeafF2 {
    float d0xh, d0xl, d0yh, d0yl;   // D0 = A + a0_x (B - A) + a0_y (C - A) - x
    float u0h, u0l, v0h, v0l;       // (u, v) = 3 a0 - 1 of the first vertex
    float sh, wjh, wjl, pad;        // sh; J_T 4^-L / 4pi
};

// The integer numerator 0 <= v <= 2^30 at scale 2^-L as an exact, normalised
// pair: h = fl(v) and l = v - h (|l| <= ulp(h) / 2).
__device__ __forceinline__ f2 dyadic_f2(int32_t v, float scale) {
    const float h = __int2float_rn(v);
    const int32_t hi = __float2int_rn(h);
    return {__fmul_rn(h, scale), __fmul_rn(__int2float_rn(v - hi), scale)};
}

// y - x at reference coordinates (xi, eta): a + xi e + eta f, per coordinate.
__device__ __forceinline__ f2 rel_coord(f2 a, f2 xi, f2 eta, f2 e, f2 f) {
    return f2_add(a, f2_add(f2_mul(xi, e), f2_mul(eta, f)));
}

// Sign decisions of the FP64 predicates taken from FP32 values when their
// error bound allows: +1/-1 decided, 0 undecided.  o = a x b for the
// vertices' offsets a, b from x (FP32 parts of float-float values accurate to
// 2^-47 relative); the bound covers the FP32 evaluation (< 2^-22 relative to
// |ax by| + |ay bx|) and the rounding of the FP64 vertex coordinates of the
// exact test (< 2^-50 cm per unit offset, cm the coordinate magnitude).
__device__ __forceinline__ int orient_filter(float ax, float ay, float bx, float by, float cm) {
    const float p1 = ax * by, p2 = ay * bx;
    const float o = p1 - p2;
    const float bound = 2.384185791015625e-07f * (fabsf(p1) + fabsf(p2)) +
                        1.7763568394002505e-15f * cm * (fabsf(ax) + fabsf(ay) + fabsf(bx) + fabsf(by));
    if (o > bound) return 1;
    if (o < -bound) return -1;
    return 0;
}

// Per-triangle, per-target and per-node data of the float-float kernels.
struct WeightsF2 {
    const float4* tA;     // [nt] A x (h, l), A y (h, l)
    const float4* te;     // [nt] (B - A) x, y
    const float4* tf;     // [nt] (C - A) x, y
    const float4* tw;     // [nt] J / 4pi (h, l), max |vertex coordinate|, 0
    const float4* x2;     // [M] target x, y
    const float4* y2;     // [N] node x, y
    const float2* wq2;    // [N] W_j / 4pi
    const double* Rn;     // [nt] near-rule ellipse parameter R = w J_T / (eps C_N) of the root
};


// Warp-wide reduce-scatter of 16 float-float values (the FP64 version's
// pattern): afterwards lane l holds the warp total of value (l >> 1).
__device__ __forceinline__ f2 reduce_scatter16_f2(f2* v, int lane) {
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const bool hi = lane & 16;
        const f2 send = hi ? v[i] : v[i + 8];
        const f2 keep = hi ? v[i + 8] : v[i];
        v[i] = f2_add(keep, {__shfl_xor_sync(0xffffffffu, send.h, 16), __shfl_xor_sync(0xffffffffu, send.l, 16)});
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const bool hi = lane & 8;
        const f2 send = hi ? v[i] : v[i + 4];
        const f2 keep = hi ? v[i + 4] : v[i];
        v[i] = f2_add(keep, {__shfl_xor_sync(0xffffffffu, send.h, 8), __shfl_xor_sync(0xffffffffu, send.l, 8)});
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool hi = lane & 4;
        const f2 send = hi ? v[i] : v[i + 2];
        const f2 keep = hi ? v[i + 2] : v[i];
        v[i] = f2_add(keep, {__shfl_xor_sync(0xffffffffu, send.h, 4), __shfl_xor_sync(0xffffffffu, send.l, 4)});
    }
    {
        const bool hi = lane & 2;
        const f2 send = hi ? v[0] : v[1];
        const f2 keep = hi ? v[1] : v[0];
        v[0] = f2_add(keep, {__shfl_xor_sync(0xffffffffu, send.h, 2), __shfl_xor_sync(0xffffffffu, send.l, 2)});
    }
    return f2_add(v[0], {__shfl_xor_sync(0xffffffffu, v[0].h, 1), __shfl_xor_sync(0xffffffffu, v[0].l, 1)});
}

// C_k = s - [k != own] W_k G(x, y_k) for node k of the pair's triangle, stored
// in FP64 and float-float.
__device__ __forceinline__ void far_subtract_store(const WeightsArgs& a, const WeightsF2& b, int64_t p, int T, int t,
                                                   int own, int k, f2 s, const float4* ftab, const LogSmem& lt,
                                                   double ln2) {
    if (k != own) {
        const int64_t j = (int64_t)T * a.nq + k;
        const float4 X = b.x2[t], Y = b.y2[j];
        const f2 dx = f2_add({X.x, X.y}, {-Y.x, -Y.y}), dy = f2_add({X.z, X.w}, {-Y.z, -Y.w});
        const f2 r2 = f2_add(f2_sqr(dx), f2_sqr(dy));
        f2 lg;
        if (r2.h > 1e-30f) ff_log(ftab, r2.h, r2.l, lg.h, lg.l);
        else lg = f2_from_d(vp_logd(f2_to_d(r2), lt.rc, lt.lc, ln2));
        const float2 wq = b.wq2[j];
        s = f2_add(s, f2_neg(f2_mul(lg, {wq.x, wq.y})));
    }
    a.C[p * a.nq + k] = f2_to_d(s);
    if (a.C2) a.C2[p * a.nq + k] = make_float2(s.h, s.l);
}

// mu_i on lanes 2i and 2i + 1 -> C_k = sum_i Q_ki mu_i - [k != own] W_k G(x, y_k)
__device__ __forceinline__ void finish_pair_mine(const WeightsArgs& a, const WeightsF2& b, int64_t p, int T, int t,
                                                 int own, f2 mine, int lane, const float4* ftab, const LogSmem& lt,
                                                 double ln2) {
    for (int k0 = 0; k0 < a.nq; k0 += 32) {   // node k0 + lane of every group of 32
        const int k = k0 + lane;
        const float2* Qk = a.Q2 + (k < a.nq ? k : 0) * VP_NB;
        float ah = 0.f, al = 0.f;     // unnormalised, as the moment accumulators
#pragma unroll
        for (int q = 0; q < VP_NB; q++) {
            const f2 mq = {__shfl_sync(0xffffffffu, mine.h, 2 * q), __shfl_sync(0xffffffffu, mine.l, 2 * q)};
            const float2 Q = Qk[q];
            f2_acc(ah, al, {Q.x, Q.y}, mq);
        }
        if (k < a.nq) far_subtract_store(a, b, p, T, t, own, k, f2_fast(ah, al), ftab, lt, ln2);
    }
}

// mu (float-float accumulators of every lane) -> the warp totals -> C_k
__device__ __forceinline__ void finish_pair_f2(const WeightsArgs& a, const WeightsF2& b, int64_t p, int T, int t,
                                               int own, const float* mh, const float* ml, int lane,
                                               const float4* ftab, const LogSmem& lt, double ln2) {
    f2 v[16];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) v[q] = f2_fast(mh[q], ml[q]);
    v[15] = {0.f, 0.f};
    finish_pair_mine(a, b, p, T, t, own, reduce_scatter16_f2(v, lane), lane, ftab, lt, ln2);
}

// Stop test of a sub-triangle S of T (vertices v) whose FP32 filters were
// undecided: x outside every edge ellipse of S (R_S = R 4^-L) and outside S,
// by the exact FP64 predicates.  Inlined: out of line (__noinline__) the
// 16,384-triangle star build took 5% longer (more spills around the call).
#ifndef VP_COLD
#define VP_COLD __forceinline__
#endif
__device__ VP_COLD bool near_stop_fp64(const double* v, SubTri S, double xx, double xy, int Nn, double R_root) {
    const double Ax = v[0], Ay = v[1];
    const double eex = rn_sub(v[2], Ax), eey = rn_sub(v[3], Ay);
    const double ffx = rn_sub(v[4], Ax), ffy = rn_sub(v[5], Ay);
    double ph[6];
    sub_phys(S, Ax, Ay, eex, eey, ffx, ffy, ph);
    return !tri_near_fast(ph, xx, xy, Nn, ldexp(R_root, -2 * S.L)) && !tri_contains_rn(ph, xx, xy);
}

// Per-pair float-float geometry of the near scheme, relative to the target.
struct NearPairF2 {
    f2 ax, ay;          // A - x
    f2 ex, ey, fx, fy;  // B - A, C - A
    f2 wj;              // J_T / 4pi
    float cm;           // coordinate magnitude bound of the orientation filter
};

__device__ __forceinline__ NearPairF2 near_pair_f2(const WeightsF2& b, int T, int t) {
    const float4 TA = b.tA[T], TE = b.te[T], TF = b.tf[T], TW = b.tw[T], X = b.x2[t];
    NearPairF2 g;
    g.ax = f2_add({TA.x, TA.y}, {-X.x, -X.y});
    g.ay = f2_add({TA.z, TA.w}, {-X.z, -X.w});
    g.ex = {TE.x, TE.y};
    g.ey = {TE.z, TE.w};
    g.fx = {TF.x, TF.y};
    g.fy = {TF.z, TF.w};
    g.wj = {TW.x, TW.y};
    g.cm = fmaxf(TW.z, fmaxf(fabsf(X.x), fabsf(X.z)));
    return g;
}

// The stop test of sub-triangle S of the pair's triangle (x outside every
// near-rule edge ellipse of S and outside S): FP32 filters on the
// float-float vertex offsets, the exact FP64 predicates when undecided.
// Also gives the leaf data: offset D0 of S's first vertex, its reference
// coordinates a0 and the scale 2^-L.
__device__ __forceinline__ bool subtri_stop_f2(const WeightsArgs& a, const NearPairF2& g, const SubTri& S, int T,
                                               int t, int Nn, double R_root, float Rf_root, float& scale, f2& d0x,
                                               f2& d0y, f2& a0x, f2& a0y) {
    scale = __int_as_float((127 - S.L) << 23);            // 2^-L
    f2 dx[3], dy[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const f2 xi = dyadic_f2(S.v[2 * i], scale), eta = dyadic_f2(S.v[2 * i + 1], scale);
        dx[i] = rel_coord(g.ax, xi, eta, g.ex, g.fx);
        dy[i] = rel_coord(g.ay, xi, eta, g.ey, g.fy);
        if (i == 0) {
            a0x = xi;
            a0y = eta;
        }
    }
    d0x = dx[0];
    d0y = dy[0];
    const float Rf = __fmul_rn(Rf_root, __fmul_rn(scale, scale));
    int near = 0;      // 1 near, 0 not near, -1 undecided
    for (int e = 0; e < 3 && near != 1; e++) {
        const int i0 = e, i1 = (e + 1) % 3;
        const int r = edge_near_f32(dx[i0].h, dy[i0].h, dx[i1].h, dy[i1].h, Nn, Rf);
        if (r == 1) near = 1;
        else if (r == 2) near = -1;
    }
    int inside = 1;    // 1 inside, 0 outside, -1 undecided
    if (near != 1) {
        for (int e = 0; e < 3 && inside != 0; e++) {
            const int i0 = e, i1 = (e + 1) % 3;
            const int o = orient_filter(dx[i0].h, dy[i0].h, dx[i1].h, dy[i1].h, g.cm);
            if (o < 0) inside = 0;
            else if (o == 0) inside = -1;
        }
    }
    if (near == 1) return false;
    if (near == 0 && inside != -1) return inside == 0;
    // undecided in FP32: the FP64 predicates on the FP64 vertices
    return near_stop_fp64(a.tv + 6 * (int64_t)T, S, a.txy[2 * t], a.txy[2 * t + 1], Nn, R_root);
}

// One (leaf, near-rule node) term: node offset D0 + sh E_j from the target,
// g = log|y - x|^2 W_j J_S / 4pi, moments += g M_ab at (u, v) = (u0, v0) +
// sh Z, Z = 3 z_j (the node's (u, v) = 3 (a0 + sh z_j) - 1).
__device__ __forceinline__ void near_leaf_node(const LeafF2& lf, float4 E, float4 Z, float2 W,
                                               const float4* ftab, const LogSmem& lt, double ln2, float* mh,
                                               float* ml) {
    const float sh = lf.sh;
    const f2 dx = f2_add({lf.d0xh, lf.d0xl}, {__fmul_rn(E.x, sh), __fmul_rn(E.y, sh)});
    const f2 dy = f2_add({lf.d0yh, lf.d0yl}, {__fmul_rn(E.z, sh), __fmul_rn(E.w, sh)});
    const f2 r2 = f2_add(f2_sqr(dx), f2_sqr(dy));
    f2 lg;
    if (r2.h > 1e-30f) ff_log(ftab, r2.h, r2.l, lg.h, lg.l);              // log |y - x|^2
    else lg = f2_from_d(vp_logd(f2_to_d(r2), lt.rc, lt.lc, ln2));        // far below any mesh scale
    const f2 g = f2_mul_u(lg, f2_mul_u({W.x, W.y}, {lf.wjh, lf.wjl}));   // only multiplied and added on
    const f2 u = f2_add({lf.u0h, lf.u0l}, {__fmul_rn(Z.x, sh), __fmul_rn(Z.y, sh)});   // Z = 3 z_j
    const f2 v = f2_add({lf.v0h, lf.v0l}, {__fmul_rn(Z.z, sh), __fmul_rn(Z.w, sh)});
    f2_mon15_acc_uv(mh, ml, g, u, v);
}

// E_j = z_j,x (B - A) + z_j,y (C - A) of the pair's triangle, per warp.
__device__ __forceinline__ void near_exy(const NearPairF2& g, const float4* nz, float4* exy, int lane) {
    for (int j = lane; j < VP_NNEAR; j += 32) {
        const float4 Z = nz[j];
        const f2 zx = {Z.x, Z.y}, zy = {Z.z, Z.w};
        const f2 Ex = f2_add(f2_mul(zx, g.ex), f2_mul(zy, g.fx)), Ey = f2_add(f2_mul(zx, g.ey), f2_mul(zy, g.fy));
        exy[j] = make_float4(Ex.h, Ex.l, Ey.h, Ey.l);
    }
}


// Near pairs whose whole triangle is already a leaf of the subdivision (about
// three in four on graded meshes) need no traversal: one thread per pair
// takes the depth-0 stop test of the traversal, writes the pair's leaf and
// capped counts when the root is a leaf, and appends the pair to the root
// list or to the list that the traversal kernel takes.
__global__ void __launch_bounds__(256) k_near_root_split(WeightsArgs a, WeightsF2 b, const int32_t* __restrict__ idx,
                                                         int64_t n, int32_t* __restrict__ root_idx,
                                                         int32_t* __restrict__ deep_idx,
                                                         unsigned long long* __restrict__ counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool root = false;
    int32_t p = 0;
    if (i < n) {
        p = idx[i];
        const int T = a.ptri[p], t = a.ptgt[p];
        const double R_root = b.Rn[T];
        const NearPairF2 g = near_pair_f2(b, T, t);
        SubTri S;
        S.v[0] = 0; S.v[1] = 0; S.v[2] = 1; S.v[3] = 0; S.v[4] = 0; S.v[5] = 1; S.L = 0;
        float scale;
        f2 d0x, d0y, a0x, a0y;
        root = subtri_stop_f2(a, g, S, T, t, a.tab->near_degree, R_root, (float)R_root, scale, d0x, d0y, a0x, a0y);
        int capped = 0;
        if (!root && a.depth_cap <= 0) {
            root = true;
            capped = 1;
        }
        if (root) {
            a.pstat[p] = 1;
            a.pcap[p] = capped;
        }
    }
    const unsigned mr = __ballot_sync(0xffffffffu, i < n && root);
    const unsigned md = __ballot_sync(0xffffffffu, i < n && !root);
    unsigned long long br = 0, bd = 0;
    if (lane == 0) {
        if (mr) br = atomicAdd(&counters[0], (unsigned long long)__popc(mr));
        if (md) bd = atomicAdd(&counters[1], (unsigned long long)__popc(md));
    }
    br = __shfl_sync(0xffffffffu, br, 0);
    bd = __shfl_sync(0xffffffffu, bd, 0);
    const unsigned lower = (1u << lane) - 1u;
    if (i < n) {
        if (root) root_idx[br + __popc(mr & lower)] = p;
        else deep_idx[bd + __popc(md & lower)] = p;
    }
}

// Root-leaf near pairs: the near rule on the whole triangle.  Its nodes sit at
// fixed reference points z_j, so the moments and the moment-to-weight map
// fold into one constant matrix of the far rule, C_k = sum_j B_jk g_j with
// g_j = log|y_j - x|^2 w_j J_T / 4pi (B = QM M(z)^T, tabulated per rule).
// A warp takes RPW pairs at once, so that its lanes stay busy: the RPW x 33
// values g_j are spread over the lanes into shared memory, then the RPW x nq
// dot products (one (pair, node) per lane) and the far-rule subtraction.
// Each (pair, node) result is computed by the same operations in the same
// order whatever lane takes it.
#ifndef VP_ROOT_MINB
#define VP_ROOT_MINB 6
#endif
#ifndef VP_ROOT_PPW
#define VP_ROOT_PPW 5
#endif
constexpr int RPW = VP_ROOT_PPW;
struct RootPair {
    NearPairF2 g;
    int32_t p, T, t, own;
};
__global__ void __launch_bounds__(WARPS * 32, VP_ROOT_MINB) k_weights_near_root(WeightsArgs a, WeightsF2 b,
                                                                                const int32_t* __restrict__ idx,
                                                                                int64_t n) {
    __shared__ float2 g_all[WARPS][RPW][VP_NNEAR];
    __shared__ RootPair rp_all[WARPS][RPW];
    __shared__ float4 ftab[LOG_N];
    __shared__ float4 nz_s[VP_NNEAR];
    __shared__ float2 nw_s[VP_NNEAR];
    __shared__ LogSmem lt;
    for (int i = threadIdx.x; i < LOG_N; i += blockDim.x) ftab[i] = g_logtab.e[i];
    for (int i = threadIdx.x; i < VP_NNEAR; i += blockDim.x) {
        nz_s[i] = a.tab->nz2[i];
        nw_s[i] = a.tab->nw2[i];
    }
    load_logtab(a.tab, lt);              // ends with __syncthreads
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const double ln2 = a.tab->ln2;
    RootPair* rp = rp_all[wl];
    // persistent: each warp takes the groups of RPW pairs at w0, w0 + RPW (warps in the grid), ...
    for (int64_t w0 = ((int64_t)blockIdx.x * WARPS + wl) * RPW; w0 < n; w0 += (int64_t)gridDim.x * WARPS * RPW) {
        const int np = (int)min((int64_t)RPW, n - w0);
        __syncwarp();
        if (lane < np) {
            RootPair r;
            r.p = idx[w0 + lane];
            r.T = a.ptri[r.p];
            r.t = a.ptgt[r.p];
            r.own = own_index(a, r.t, r.T);
            r.g = near_pair_f2(b, r.T, r.t);
            rp[lane] = r;
        }
        __syncwarp();
        for (int e = lane; e < np * VP_NNEAR; e += 32) {
            const int q = e / VP_NNEAR, j = e - q * VP_NNEAR;
            const NearPairF2 g = rp[q].g;
            const float4 Z = nz_s[j];
            const f2 zx = {Z.x, Z.y}, zy = {Z.z, Z.w};
            const f2 dx = f2_add(g.ax, f2_add(f2_mul(zx, g.ex), f2_mul(zy, g.fx)));   // y_j - x
            const f2 dy = f2_add(g.ay, f2_add(f2_mul(zx, g.ey), f2_mul(zy, g.fy)));
            const f2 r2 = f2_add(f2_sqr(dx), f2_sqr(dy));
            f2 lg;
            if (r2.h > 1e-30f) ff_log(ftab, r2.h, r2.l, lg.h, lg.l);
            else lg = f2_from_d(vp_logd(f2_to_d(r2), lt.rc, lt.lc, ln2));
            const float2 W = nw_s[j];
            const f2 gj = f2_mul_u(lg, f2_mul_u({W.x, W.y}, g.wj));   // a factor of the products below
            g_all[wl][q][j] = make_float2(gj.h, gj.l);
        }
        __syncwarp();
        for (int sl = lane; sl < np * a.nq; sl += 32) {
            const int q = sl / a.nq, k = sl - q * a.nq;
            const float2* gs = g_all[wl][q];
            const float2* Bk = a.B2 + k;
            float ah = 0.f, al = 0.f;
#pragma unroll 11
            for (int j = 0; j < VP_NNEAR; j++) {
                const float2 gj = gs[j], B = Bk[(int64_t)j * a.nq];
                f2_acc(ah, al, {B.x, B.y}, {gj.x, gj.y});
                if ((j & 7) == 7) {
                    const f2 r = f2_fast(ah, al);
                    ah = r.h;
                    al = r.l;
                }
            }
            const RootPair& r = rp[q];
            far_subtract_store(a, b, r.p, r.T, r.t, r.own, k, f2_fast(ah, al), ftab, lt, ln2);
        }
    }
}

// Near pairs whose root is not a leaf, in three steps.  One thread per pair
// runs the subdivision depth first from the root's four children with the
// traversal's stop test, counting its leaves (pass 0) and, after a scan,
// writing them (pass 1) as (first vertex, level, orientation) records; then a
// warp per pair evaluates its leaves 32 at a time (k_weights_near_deep).
struct LeafRec {
    int32_t x, y;    // first vertex, numerators at scale 2^-L
    int32_t L;
    int32_t flip;    // 1: the inverted child (m12, m20, m01), sh = -2^-L
};
// Per-thread stack of the depth-first subdivision: 3 entries per level of
// depth + 4 (depth cap 30), 12 bytes each.  Every sub-triangle of the 4-way
// midpoint split is a right triangle of the reference simplex with legs of
// one unit at its scale 2^-L, upright, (x, y), (x + 1, y), (x, y + 1), or
// inverted, (x, y), (x - 1, y), (x, y - 1), so its first vertex, level and
// orientation determine it.
constexpr int DSTK = 96;
struct StackRec {
    int32_t x, y;    // first vertex, numerators at scale 2^-L
    int32_t lf;      // 2 L + (1: inverted)
};

__device__ __forceinline__ SubTri stack_subtri(StackRec r) {
    const int32_t sg = (r.lf & 1) ? -1 : 1;
    SubTri S;
    S.v[0] = r.x; S.v[1] = r.y; S.v[2] = r.x + sg; S.v[3] = r.y; S.v[4] = r.x; S.v[5] = r.y + sg;
    S.L = r.lf >> 1;
    return S;
}

// The four children of r in push_children's order: (v0, m01, m20),
// (m01, v1, m12), (m20, m12, v2) keep the orientation, (m12, m20, m01) flips it.
__device__ __forceinline__ void push_children_rec(StackRec r, StackRec* stk, int base) {
    const int32_t sg = (r.lf & 1) ? -1 : 1, lf = r.lf + 2;
    stk[base + 0] = {2 * r.x, 2 * r.y, lf};
    stk[base + 1] = {2 * r.x + sg, 2 * r.y, lf};
    stk[base + 2] = {2 * r.x, 2 * r.y + sg, lf};
    stk[base + 3] = {2 * r.x + sg, 2 * r.y + sg, lf ^ 1};
}

__global__ void __launch_bounds__(128) k_near_deep_leaves(WeightsArgs a, WeightsF2 b, const int32_t* __restrict__ idx,
                                                          int64_t n, int pass, int32_t* __restrict__ cnt,
                                                          const int64_t* __restrict__ off, LeafRec* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = idx[i];
    const int T = a.ptri[p], t = a.ptgt[p];
    const int Nn = a.tab->near_degree;
    const double R_root = b.Rn[T];
    const float Rf_root = (float)R_root;
    const NearPairF2 g = near_pair_f2(b, T, t);
    StackRec stk[DSTK];
    push_children_rec({0, 0, 0}, stk, 0);
    int sp = 4, capped = 0, visited = 1;
    int64_t nleaf = 0;
    bool overflow = false;
    const int64_t base = pass ? off[i] : 0;
    while (sp > 0) {
        if (++visited > MAX_VISITED) {
            overflow = true;
            break;
        }
        const StackRec R = stk[--sp];
        const SubTri S = stack_subtri(R);
        float scale;
        f2 d0x, d0y, a0x, a0y;
        bool stop = subtri_stop_f2(a, g, S, T, t, Nn, R_root, Rf_root, scale, d0x, d0y, a0x, a0y);
        if (!stop && S.L >= a.depth_cap) {
            stop = true;
            capped++;
        }
        if (stop) {
            if (pass) {
                LeafRec lr;
                lr.x = S.v[0];
                lr.y = S.v[1];
                lr.L = S.L;
                lr.flip = (S.v[2] - S.v[0]) > 0 ? 0 : 1;
                out[base + nleaf] = lr;
            }
            nleaf++;
        } else {
            if (sp + 4 > DSTK) {
                overflow = true;
                break;
            }
            push_children_rec(R, stk, sp);
            sp += 4;
        }
    }
    if (overflow) atomicOr(a.flag, VP_DEV_ERR_STACK);
    if (pass == 0) {
        cnt[i] = (int32_t)nleaf;
    } else {
        a.pstat[p] = (int32_t)nleaf;
        a.pcap[p] = capped;
    }
}

#ifndef VP_DEEP_MINB
#define VP_DEEP_MINB 5
#endif
__global__ void __launch_bounds__(WARPS * 32, VP_DEEP_MINB) k_weights_near_deep(WeightsArgs a, WeightsF2 b,
                                                                                const int32_t* __restrict__ idx,
                                                                                int64_t n,
                                                                                const int64_t* __restrict__ off,
                                                                                const LeafRec* __restrict__ recs) {
    __shared__ LeafF2 leaf_all[WARPS][32];
    __shared__ float4 exy_all[WARPS][VP_NNEAR];
    __shared__ float4 ftab[LOG_N];
    __shared__ float4 nz_s[VP_NNEAR];
    __shared__ float4 nz3_s[VP_NNEAR];   // 3 z_j, float-float
    __shared__ float2 nw_s[VP_NNEAR];
    __shared__ LogSmem lt;
    for (int i = threadIdx.x; i < LOG_N; i += blockDim.x) ftab[i] = g_logtab.e[i];
    for (int i = threadIdx.x; i < VP_NNEAR; i += blockDim.x) {
        nz_s[i] = a.tab->nz2[i];
        nz3_s[i] = a.tab->nz3[i];
        nw_s[i] = a.tab->nw2[i];
    }
    load_logtab(a.tab, lt);              // ends with __syncthreads
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const double ln2 = a.tab->ln2;
    LeafF2* leaves = leaf_all[wl];
    float4* exy = exy_all[wl];
    // persistent: each warp takes pairs w, w + (warps in the grid), ...
    for (int64_t w = (int64_t)blockIdx.x * WARPS + wl; w < n; w += (int64_t)gridDim.x * WARPS) {
        __syncwarp();
        const int64_t p = idx[w];
        const int T = a.ptri[p], t = a.ptgt[p];
        const int own = own_index(a, t, T);
        const NearPairF2 g = near_pair_f2(b, T, t);
        near_exy(g, nz_s, exy, lane);
        float mh[VP_NB], ml[VP_NB];
#pragma unroll
        for (int q = 0; q < VP_NB; q++) mh[q] = ml[q] = 0.f;
        const int64_t l0 = off[w], l1 = off[w + 1];
        for (int64_t c0 = l0; c0 < l1; c0 += 32) {
            const int nl = (int)min((int64_t)32, l1 - c0);
            __syncwarp();
            if (lane < nl) {
                // the leaf data exactly as the traversal forms it (subtri_stop_f2)
                const LeafRec lr = recs[c0 + lane];
                const float scale = __int_as_float((127 - lr.L) << 23);
                const f2 xi = dyadic_f2(lr.x, scale), eta = dyadic_f2(lr.y, scale);
                const f2 d0x = rel_coord(g.ax, xi, eta, g.ex, g.fx), d0y = rel_coord(g.ay, xi, eta, g.ey, g.fy);
                const f2 u0 = f2_axpb(xi, 3.0f, -1.0f), v0 = f2_axpb(eta, 3.0f, -1.0f);
                const f2 wj = f2_scale(g.wj, __fmul_rn(scale, scale));
                LeafF2 lf;
                lf.d0xh = d0x.h; lf.d0xl = d0x.l; lf.d0yh = d0y.h; lf.d0yl = d0y.l;
                lf.u0h = u0.h; lf.u0l = u0.l; lf.v0h = v0.h; lf.v0l = v0.l;
                lf.sh = lr.flip ? -scale : scale;
                lf.wjh = wj.h; lf.wjl = wj.l; lf.pad = 0.f;
                leaves[lane] = lf;
            }
            __syncwarp();
            const int combos = nl * VP_NNEAR;
            for (int i = lane; i < combos; i += 32) {
                const int li = i / VP_NNEAR, j = i - li * VP_NNEAR;
                near_leaf_node(leaves[li], exy[j], nz3_s[j], nw_s[j], ftab, lt, ln2, mh, ml);
            }
        }
        finish_pair_f2(a, b, p, T, t, own, mh, ml, lane, ftab, lt, ln2);
    }
}

// ---------------------------------------------------- self, float-float
// Section 3.4: the fan of the target over each side of T, panels dyadic
// towards the foot of the perpendicular, a Gauss-Legendre rule in arc length
// per panel and a radial rule along each ray.  The per-edge geometry that
// fixes the panels (side lengths, the foot of the perpendicular, the
// distance to the side, the dyadic panel counts) is FP64 exactly as in the
// FP64 kernel; everything per panel in float-float.
//
// Along the ray from the target x to the boundary point gamma(s) at distance
// r0, the point at fraction r has (u, v) = (u0, v0) + r (al, be), so each
// monomial u^a v^b of the P_4 moments is a polynomial of degree <= 4 in r and
// the radial integrand is r log(r r0) times it.  The interpolatory rule on
// the 5 Gauss-Legendre nodes of [0, 1] with the weights of int r p and
// int r log(r) p (vp_tables.h) is exact for these, as the paper's
// generalized Gaussian rule of order 8 is: the moments are the same up to
// rounding, with one logarithm per ray and 5 points instead of 8.
// Lanes: Gauss-Legendre node lane & 15 of panel 2 i + (lane >> 4).
__device__ __forceinline__ f2 self_bound(int k, int Nd, int side, f2 L2, f2 st2, f2 len2) {
    if (k == 0) return side == 0 ? f2{0.f, 0.f} : L2;           // the side's end
    if (k == Nd + 1) return st2;                                  // the foot
    const f2 om = k <= 24 ? f2{__fsub_rn(1.f, __int_as_float((127 - k) << 23)), 0.f}   // 1 - 2^-k, exact
                          : f2{1.f, -__int_as_float((127 - min(k, 126)) << 23)};
    const f2 frac = f2_mul(len2, om);
    return side == 0 ? frac : f2_add(L2, f2_neg(frac));
}

__global__ void __launch_bounds__(WARPS * 32, VP_SELF_MINB) k_weights_self_f2(WeightsArgs a, WeightsF2 b,
                                                                              const int32_t* __restrict__ idx,
                                                                              int64_t n) {
    __shared__ float4 ftab[LOG_N];
    __shared__ LogSmem lt;
    load_logtab(a.tab, lt);
    for (int i = threadIdx.x; i < LOG_N; i += blockDim.x) ftab[i] = g_logtab.e[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (w >= n) return;
    const double ln2 = a.tab->ln2;
    const int64_t p = idx[w];
    const int T = a.ptri[p], t = a.ptgt[p];
    const double* v = a.tv + 6 * (int64_t)T;
    const double Ax = v[0], Ay = v[1];
    const double ex = v[2] - Ax, ey = v[3] - Ay, fx = v[4] - Ax, fy = v[5] - Ay;
    const double invJ = 1.0 / a.J[T];
    const double xx = a.txy[2 * t], xy = a.txy[2 * t + 1];
    const double qx0 = xx - Ax, qy0 = xy - Ay;
    const f2 xi0 = f2_from_d((qx0 * fy - qy0 * fx) * invJ), eta0 = f2_from_d((ex * qy0 - ey * qx0) * invJ);
    const int own = own_index(a, t, T);
    // float-float triangle relative to the target
    const float4 TA = b.tA[T], TE = b.te[T], TF = b.tf[T], X = b.x2[t];
    const f2 ax = f2_add({TA.x, TA.y}, {-X.x, -X.y}), ay = f2_add({TA.z, TA.w}, {-X.z, -X.w});
    const f2 e2x = {TE.x, TE.y}, e2y = {TE.z, TE.w}, f2x = {TF.x, TF.y}, f2y = {TF.z, TF.w};
    const int gl = lane & 15, half = lane >> 4;
    const float2 LX = a.tab->lx2[gl], LW = a.tab->lw2[gl];
    const f2 lx = {LX.x, LX.y}, lw = {LW.x, LW.y};
    // The three sides' FP64 geometry, side e on lane e (the FP64 pipe is
    // charged per warp instruction: one instruction serves all three sides).
    double gL = 0.0, gh = 0.0;
    f2 ginvL = {0.f, 0.f}, gst = {0.f, 0.f};
    int gnd0 = -1, gnd1 = -1;            // -1: no panels on that half of the side
    if (lane < 3) {
        const int e = lane;
        const double Px = v[2 * e], Py = v[2 * e + 1];
        const double Qx = v[(2 * e + 2) % 6], Qy = v[(2 * e + 3) % 6];
        const double dx = rn_sub(Qx, Px), dy = rn_sub(Qy, Py);
        gL = rn_sqrt(rn_add(rn_mul(dx, dx), rn_mul(dy, dy)));
        if (gL != 0.0) gh = rn_div(fabs(rn_sub(rn_mul(dx, rn_sub(xy, Py)), rn_mul(dy, rn_sub(xx, Px)))), gL);
        if (gL != 0.0 && gh != 0.0) {
            double st = rn_div(rn_add(rn_mul(dx, rn_sub(xx, Px)), rn_mul(dy, rn_sub(xy, Py))), gL);
            if (st < 0.0) st = 0.0;
            if (st > gL) st = gL;
            const double fxp = rn_add(Px, rn_mul(rn_div(st, gL), dx)), fyp = rn_add(Py, rn_mul(rn_div(st, gL), dy));
            const double ddx = rn_sub(xx, fxp), ddy = rn_sub(xy, fyp);
            const double delta = rn_sqrt(rn_add(rn_mul(ddx, ddx), rn_mul(ddy, ddy)));
            const double Lst = rn_sub(gL, st);
            gnd0 = st > 0.0 ? dyadic_count(st, delta) : -1;
            gnd1 = Lst > 0.0 ? dyadic_count(Lst, delta) : -1;
            ginvL = f2_from_d(1.0 / gL);
            gst = f2_from_d(st);
        }
    }
    const f2 gL2 = f2_from_d(gL), gh2 = f2_from_d(gh);
    // panels of the six (side, half) segments, in the order side 0 half 0, ...
    int cnt[6], total = 0;
#pragma unroll
    for (int e = 0; e < 3; e++) {
        cnt[2 * e] = __shfl_sync(0xffffffffu, gnd0, e) + 1;
        cnt[2 * e + 1] = __shfl_sync(0xffffffffu, gnd1, e) + 1;
        total += cnt[2 * e] + cnt[2 * e + 1];
    }
    const f2 u0 = f2_axpb(xi0, 3.0f, -1.0f), v0 = f2_axpb(eta0, 3.0f, -1.0f);   // the target's (u, v)
    float mh[VP_NB], ml[VP_NB];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) mh[q] = ml[q] = 0.f;
    for (int pb = 0; pb < total; pb += 2) {
        const int pi = pb + half;
        const bool active = pi < total;
        int i = active ? pi : total - 1, seg = 0, Nd = cnt[0] - 1;
#pragma unroll
        for (int k = 0; k < 5; k++)            // the segment of panel i (static indices: registers)
            if (seg == k && i >= cnt[k]) {
                i -= cnt[k];
                seg = k + 1;
                Nd = cnt[k + 1] - 1;
            }
        const int e = seg >> 1, side = seg & 1;
        const f2 L2 = {__shfl_sync(0xffffffffu, gL2.h, e), __shfl_sync(0xffffffffu, gL2.l, e)};
        const f2 h2 = {__shfl_sync(0xffffffffu, gh2.h, e), __shfl_sync(0xffffffffu, gh2.l, e)};
        const f2 invL = {__shfl_sync(0xffffffffu, ginvL.h, e), __shfl_sync(0xffffffffu, ginvL.l, e)};
        const f2 st2 = {__shfl_sync(0xffffffffu, gst.h, e), __shfl_sync(0xffffffffu, gst.l, e)};
        if (!active) continue;
        // the side in float-float: P - x, Q - P, and in reference coordinates
        const f2 pxr = e == 0 ? ax : f2_add(ax, e == 1 ? e2x : f2x);
        const f2 pyr = e == 0 ? ay : f2_add(ay, e == 1 ? e2y : f2y);
        const f2 sdx = e == 0 ? e2x : (e == 1 ? f2_add(f2x, f2_neg(e2x)) : f2_neg(f2x));
        const f2 sdy = e == 0 ? e2y : (e == 1 ? f2_add(f2y, f2_neg(e2y)) : f2_neg(f2y));
        const float pref_x = e == 1 ? 1.f : 0.f, pref_y = e == 2 ? 1.f : 0.f;        // P in T's simplex
        const float dref_x = e == 0 ? 1.f : (e == 1 ? -1.f : 0.f);                   // Q - P there
        const float dref_y = e == 0 ? 0.f : (e == 1 ? 1.f : -1.f);
        const f2 xiP = f2_add_f(f2_neg(xi0), pref_x), etaP = f2_add_f(f2_neg(eta0), pref_y);   // P - x, reference
        const f2 len2 = side == 0 ? st2 : f2_add(L2, f2_neg(st2));
        const f2 b0 = self_bound(i, Nd, side, L2, st2, len2), b1 = self_bound(i + 1, Nd, side, L2, st2, len2);
        const f2 D = f2_add(b1, f2_neg(b0));
        const f2 s = f2_add(b0, f2_mul(D, lx));
        f2 wd = f2_mul(D, lw);
        if (wd.h < 0.f) wd = f2_neg(wd);
        const f2 ws = f2_mul(wd, h2);
        const f2 sl = f2_mul(s, invL);
        const f2 rx = f2_add(pxr, f2_mul(sl, sdx)), ry = f2_add(pyr, f2_mul(sl, sdy));
        const f2 r2 = f2_add(f2_sqr(rx), f2_sqr(ry));
        f2 lg;
        if (r2.h > 1e-30f) ff_log(ftab, r2.h, r2.l, lg.h, lg.l);
        else lg = f2_from_d(vp_logd(f2_to_d(r2), lt.rc, lt.lc, ln2));
        const f2 lr0 = f2_scale(lg, 0.5f);                                // log r0
        const f2 al = f2_mulf(f2_add(xiP, f2_scale(sl, dref_x)), 3.0f);   // (u, v) = (u0, v0) + r (al, be)
        const f2 be = f2_mulf(f2_add(etaP, f2_scale(sl, dref_y)), 3.0f);
#pragma unroll 1
        for (int q = 0; q < VP_NRAD; q++) {   // not unrolled: the body stays in the instruction cache
            const float2 R = a.tab->rr2[q], A = a.tab->ra2[q], B = a.tab->rb2[q];
            // products that are only added or multiplied on stay unnormalised
            const f2 g = f2_mul_u(ws, f2_add(f2_mul_u(lr0, {A.x, A.y}), {B.x, B.y}));
            f2_mon15_acc_uv(mh, ml, g, f2_add(f2_mul_u({R.x, R.y}, al), u0), f2_add(f2_mul_u({R.x, R.y}, be), v0));
        }
    }
    finish_pair_f2(a, b, p, T, t, own, mh, ml, lane, ftab, lt, ln2);
    if (lane == 0) {
        a.pstat[p] = total;
        a.pcap[p] = 0;
    }
}

// float-float geometry of the weights kernels
__global__ void k_weights_f2_tri(const double* __restrict__ tv, const double* __restrict__ J, int64_t nt,
                                 float4* __restrict__ tA, float4* __restrict__ te, float4* __restrict__ tf,
                                 float4* __restrict__ tw, const VpTables* __restrict__ tab, double eps,
                                 double cn, double* __restrict__ Rn) {
    const int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= nt) return;
    const double* v = tv + 6 * T;
    const f2 Ax = f2_from_d(v[0]), Ay = f2_from_d(v[1]);
    const f2 ex = f2_from_d(rn_sub(v[2], v[0])), ey = f2_from_d(rn_sub(v[3], v[1]));
    const f2 fx = f2_from_d(rn_sub(v[4], v[0])), fy = f2_from_d(rn_sub(v[5], v[1]));
    const f2 wj = f2_from_d(J[T] * (0.5 * VP_INV_TWO_PI));
    double cm = 0.0;
    for (int i = 0; i < 6; i++) cm = fmax(cm, fabs(v[i]));
    tA[T] = make_float4(Ax.h, Ax.l, Ay.h, Ay.l);
    te[T] = make_float4(ex.h, ex.l, ey.h, ey.l);
    tf[T] = make_float4(fx.h, fx.l, fy.h, fy.l);
    tw[T] = make_float4(wj.h, wj.l, (float)(cm * 1.0000001), 0.f);
    Rn[T] = ellipse_R_rn(tab->near_what, J[T], eps, cn);
}

__global__ void k_weights_f2_pts(const double* __restrict__ xy, int64_t n, const double* __restrict__ W,
                                 float4* __restrict__ out, float2* __restrict__ wq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const f2 x = f2_from_d(xy[2 * i]), y = f2_from_d(xy[2 * i + 1]);
    out[i] = make_float4(x.h, x.l, y.h, y.l);
    if (W) {
        const f2 w = f2_from_d(W[i] * (0.5 * VP_INV_TWO_PI));
        wq[i] = make_float2(w.h, w.l);
    }
}

}  // namespace

size_t weights_f2_bytes(int64_t nt, int64_t M, int64_t N, int64_t n_near) {
    // eight arrays, the two near-pair lists and their counters, each rounded up to 256 bytes
    return (size_t)nt * (4 * sizeof(float4) + sizeof(double)) + (size_t)M * sizeof(float4) +
           (size_t)N * (sizeof(float4) + sizeof(float2)) + (size_t)n_near * 2 * sizeof(int32_t) +
           2 * sizeof(unsigned long long) + 11 * 256;
}

// float-float triangles, targets and nodes in the caller's scratch; ws
// points past them on return
static WeightsF2 weights_f2_prepare(const WeightsArgs& a, cudaStream_t s, char*& ws) {
    ws = (char*)a.f2_ws;
    auto take = [&](size_t bytes) {
        char* p = ws;
        ws += (bytes + 255) & ~(size_t)255;
        return p;
    };
    WeightsF2 b;
    float4* tA = (float4*)take(a.nt * sizeof(float4));
    float4* te = (float4*)take(a.nt * sizeof(float4));
    float4* tf = (float4*)take(a.nt * sizeof(float4));
    float4* tw = (float4*)take(a.nt * sizeof(float4));
    float4* x2 = (float4*)take(a.M * sizeof(float4));
    float4* y2 = (float4*)take(a.N * sizeof(float4));
    float2* wq2 = (float2*)take(a.N * sizeof(float2));
    double* Rn = (double*)take(a.nt * sizeof(double));
    if (a.nt > 0)
        k_weights_f2_tri<<<(unsigned)((a.nt + 255) / 256), 256, 0, s>>>(a.tv, a.J, a.nt, tA, te, tf, tw, a.tab, a.eps,
                                                                      a.c_near, Rn);
    if (a.M > 0) k_weights_f2_pts<<<(unsigned)((a.M + 255) / 256), 256, 0, s>>>(a.txy, a.M, nullptr, x2, nullptr);
    if (a.N > 0) k_weights_f2_pts<<<(unsigned)((a.N + 255) / 256), 256, 0, s>>>(a.y, a.N, a.W, y2, wq2);
    b.tA = tA; b.te = te; b.tf = tf; b.tw = tw; b.x2 = x2; b.y2 = y2; b.wq2 = wq2; b.Rn = Rn;
    return b;
}

static __global__ void k_set_flag(int32_t* flag, int32_t bits) { atomicOr(flag, bits); }

// Resident blocks per SM of the persistent weight kernels (weights_module_prepare).
static struct {
    int deep = 1, root = 1;
} g_occ;

// Blocks of a persistent launch over n units, per_block units a block: no
// more than fill the GPU once.
static unsigned persistent_grid(const vp_ctx* ctx, int64_t n, int per_block, int occ) {
    const int64_t need = (n + per_block - 1) / per_block;
    const int64_t full = (int64_t)std::max(ctx->sm_count, 1) * std::max(occ, 1);
    return (unsigned)std::max<int64_t>(1, std::min(need, full));
}

// The deep near pairs: leaf counts, their scan, the leaf records, the
// evaluation (k_near_deep_leaves, k_weights_near_deep).
static void near_deep(const WeightsArgs& a, const WeightsF2& b, const int32_t* deep_idx, int64_t n_deep, cudaStream_t s,
                      vp_ctx* ctx) {
    int32_t* cnt = nullptr;
    int64_t* off = nullptr;
    LeafRec* recs = nullptr;
    if (cudaMalloc(&cnt, n_deep * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&off, (n_deep + 1) * sizeof(int64_t)) != cudaSuccess) {
        k_set_flag<<<1, 1, 0, s>>>(a.flag, VP_DEV_ERR_ALLOC);
        cudaFree(cnt);
        cudaFree(off);
        return;
    }
    const unsigned gt = (unsigned)((n_deep + 127) / 128);
    k_near_deep_leaves<<<gt, 128, 0, s>>>(a, b, deep_idx, n_deep, 0, cnt, nullptr, nullptr);
    int64_t total = 0;
    if (vp_exclusive_scan_i32(ctx, cnt, off, n_deep, s) == VP_OK &&
        cudaMemcpyAsync(&total, off + n_deep, sizeof(int64_t), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess &&
        cudaMalloc(&recs, std::max<int64_t>(total, 1) * sizeof(LeafRec)) == cudaSuccess) {
        k_near_deep_leaves<<<gt, 128, 0, s>>>(a, b, deep_idx, n_deep, 1, cnt, off, recs);
        k_weights_near_deep<<<persistent_grid(ctx, n_deep, WARPS, g_occ.deep), WARPS * 32, 0, s>>>(a, b, deep_idx,
                                                                                                   n_deep, off, recs);
    } else {
        k_set_flag<<<1, 1, 0, s>>>(a.flag, VP_DEV_ERR_ALLOC);
    }
    cudaStreamSynchronize(s);
    cudaFree(recs);
    cudaFree(cnt);
    cudaFree(off);
}

void launch_weights(const WeightsArgs& a, const int32_t* self_idx, int64_t n_self, const int32_t* near_idx,
                    int64_t n_near, cudaStream_t s, vp_ctx* ctx) {
    const unsigned gs = (unsigned)((n_self + WARPS - 1) / WARPS), gn = (unsigned)((n_near + WARPS - 1) / WARPS);
    if (a.fp64) {
        PROF(ctx, ST_WEIGHTS_SELF, s, if (n_self > 0) k_weights_self<<<gs, WARPS * 32, 0, s>>>(a, self_idx, n_self));
        PROF(ctx, ST_WEIGHTS_NEAR, s, if (n_near > 0) k_weights_near<<<gn, WARPS * 32, 0, s>>>(a, near_idx, n_near));
        return;
    }
    ensure_logtab();
    char* ws = nullptr;
    const WeightsF2 b = weights_f2_prepare(a, s, ws);
    PROF(ctx, ST_WEIGHTS_SELF, s, if (n_self > 0) k_weights_self_f2<<<gs, WARPS * 32, 0, s>>>(a, b, self_idx, n_self));
    if (n_near <= 0) return;
    auto take = [&](size_t bytes) {
        char* q = ws;
        ws += (bytes + 255) & ~(size_t)255;
        return q;
    };
    int32_t* root_idx = (int32_t*)take(n_near * sizeof(int32_t));
    int32_t* deep_idx = (int32_t*)take(n_near * sizeof(int32_t));
    unsigned long long* cnt = (unsigned long long*)take(2 * sizeof(unsigned long long));
    unsigned long long h_cnt[2] = {0, 0};
    PROF(ctx, ST_WEIGHTS_NEAR, s, {
        cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s);
        k_near_root_split<<<(unsigned)((n_near + 255) / 256), 256, 0, s>>>(a, b, near_idx, n_near, root_idx, deep_idx,
                                                                           cnt);
        cudaMemcpyAsync(h_cnt, cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        const int64_t n_root = (int64_t)h_cnt[0], n_deep = (int64_t)h_cnt[1];
        if (n_root > 0)
            k_weights_near_root<<<persistent_grid(ctx, n_root, WARPS * RPW, g_occ.root), WARPS * 32, 0, s>>>(
                a, b, root_idx, n_root);
        if (n_deep > 0) near_deep(a, b, deep_idx, n_deep, s, ctx);
    });
}

// Loads this unit's log table on the current device (vp_create).
cudaError_t weights_module_prepare() {
    cudaError_t e = ensure_logtab();
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ.deep, k_weights_near_deep, WARPS * 32, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ.root, k_weights_near_root, WARPS * 32, 0);
    return e;
}
