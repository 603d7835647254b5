// Correction weights for (target, triangle) pairs: FP64, one warp per pair.
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
// The kernels are bound by the FP64 pipe, so per quadrature point they
// accumulate the moments mu_i of the tensor-Legendre basis leg15 (20 FP64
// operations instead of ~60 for the orthonormal basis) and use the
// table-driven vp_logd; the constant matrix Q (generated in high precision)
// maps mu to the nodal weights: C_k = sum_i Q_ki mu_i - [k != own] W_k G.
#include "vp_internal.h"

namespace {

constexpr int WARPS = 4;
constexpr int STK = 256;      // sub-triangle stack per warp
constexpr int LEAFCAP = 64;   // leaf buffer per warp
constexpr int MAX_VISITED = 1 << 20;  // sub-triangles per pair before giving up with an error flag


// Reduce-scatter of 16 per-lane values over the warp: after the five steps
// lane l holds the warp total of value (l >> 1) (16 + 8 + 4 + 2 + 1 adds
// instead of 5 x 15 for a butterfly of every value).
__device__ __forceinline__ double reduce_scatter16(double* v, int lane) {
    // step with offset 16: keep the half selected by bit 4 of the lane
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const bool hi = lane & 16;
        const double send = hi ? v[i] : v[i + 8];
        const double keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const bool hi = lane & 8;
        const double send = hi ? v[i] : v[i + 4];
        const double keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool hi = lane & 4;
        const double send = hi ? v[i] : v[i + 2];
        const double keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        const double send = hi ? v[0] : v[1];
        const double keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// mu_i -> C_k for lanes k < nq, written to C[p*nq + k].
__device__ __forceinline__ void finish_pair(const WeightsArgs& a, int64_t p, int T, int own, double xx, double xy,
                                            double* m, int lane, const double* rc, const double* lc, double ln2) {
    double v[16];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) v[q] = m[q];
    v[15] = 0.0;
    // index held by this lane after the reduce-scatter: bits 4..1 of the lane
    const double mine = reduce_scatter16(v, lane);
    double s = 0.0;
    const double* Qk = a.tab->Q[a.rule][lane < a.nq ? lane : 0];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) s = fma(Qk[q], __shfl_sync(0xffffffffu, mine, 2 * q), s);
    if (lane < a.nq) {
        if (lane != own) {
            const int64_t j = (int64_t)T * a.nq + lane;
            const double dx = xx - a.y[2 * j], dy = xy - a.y[2 * j + 1];
            s -= a.W[j] * (vp_logd(dx * dx + dy * dy, rc, lc, ln2) * (0.5 * VP_INV_TWO_PI));
        }
        a.C[p * a.nq + lane] = s;
    }
}

__device__ __forceinline__ int own_index(const WeightsArgs& a, int t, int T) {
    int tn = a.tnode[t];
    return (tn >= 0 && tn / a.nq == T) ? tn - T * a.nq : -1;
}

struct LogSmem {
    double rc[128], lc[128];
};

__device__ __forceinline__ void load_logtab(const VpTables* tab, LogSmem& t) {
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        t.rc[i] = tab->log_rc[i];
        t.lc[i] = tab->log_lc[i];
    }
    __syncthreads();
}

__device__ __forceinline__ void accumulate(double* m, double g, double x, double y) {
    double L[VP_NB];
    leg15(x, y, L);
    m[0] += g;
#pragma unroll
    for (int c = 1; c < VP_NB; c++) m[c] = fma(g, L[c], m[c]);
}

// N = min{n >= 0 : 2^-n len < dist}
__device__ __forceinline__ int dyadic_count(double len, double dist) {
    int n = 0;
    while (ldexp(len, -n) >= dist && n < 1100) n++;
    return n;
}

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
struct SubTri {
    int32_t v[6];  // vertex numerators in the reference simplex of T, at scale 2^-L
    int32_t L;
};

// A leaf as its affine map from the near rule's simplex to T's reference
// simplex (xi = a0 + zx e1 + zy e2) and its weight factor J_S / (4 pi).
struct LeafMap {
    double a0x, a0y, e1x, e1y, e2x, e2y, wJ;
};

__device__ __forceinline__ void sub_phys(const SubTri& S, double Ax, double Ay, double ex, double ey, double fx,
                                         double fy, double* ph) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double xi = ldexp((double)S.v[2 * i], -S.L), eta = ldexp((double)S.v[2 * i + 1], -S.L);
        ph[2 * i] = rn_add(Ax, rn_add(rn_mul(xi, ex), rn_mul(eta, fx)));
        ph[2 * i + 1] = rn_add(Ay, rn_add(rn_mul(xi, ey), rn_mul(eta, fy)));
    }
}

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
    const double what = a.tab->near_what;
    const int Nn = a.tab->near_degree;
    const double R_root = ellipse_R_rn(what, J, a.eps, a.c_near);
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
                    const int base = sp + 4 * __popc(sm & lower);
                    int32_t m01x = S.v[0] + S.v[2], m01y = S.v[1] + S.v[3];
                    int32_t m12x = S.v[2] + S.v[4], m12y = S.v[3] + S.v[5];
                    int32_t m20x = S.v[4] + S.v[0], m20y = S.v[5] + S.v[1];
                    int32_t V0x = 2 * S.v[0], V0y = 2 * S.v[1], V1x = 2 * S.v[2], V1y = 2 * S.v[3];
                    int32_t V2x = 2 * S.v[4], V2y = 2 * S.v[5];
                    const int32_t L1 = S.L + 1;
                    SubTri ch;
                    ch.L = L1;
                    ch.v[0] = V0x; ch.v[1] = V0y; ch.v[2] = m01x; ch.v[3] = m01y; ch.v[4] = m20x; ch.v[5] = m20y;
                    stack[base + 0] = ch;
                    ch.v[0] = m01x; ch.v[1] = m01y; ch.v[2] = V1x; ch.v[3] = V1y; ch.v[4] = m12x; ch.v[5] = m12y;
                    stack[base + 1] = ch;
                    ch.v[0] = m20x; ch.v[1] = m20y; ch.v[2] = m12x; ch.v[3] = m12y; ch.v[4] = V2x; ch.v[5] = V2y;
                    stack[base + 2] = ch;
                    ch.v[0] = m12x; ch.v[1] = m12y; ch.v[2] = m20x; ch.v[3] = m20y; ch.v[4] = m01x; ch.v[5] = m01y;
                    stack[base + 3] = ch;
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

}  // namespace

void launch_weights_self(const WeightsArgs& a, const int32_t* idx, int64_t n, cudaStream_t s) {
    if (n > 0) k_weights_self<<<(unsigned)((n + WARPS - 1) / WARPS), WARPS * 32, 0, s>>>(a, idx, n);
}

void launch_weights_near(const WeightsArgs& a, const int32_t* idx, int64_t n, cudaStream_t s) {
    if (n > 0) k_weights_near<<<(unsigned)((n + WARPS - 1) / WARPS), WARPS * 32, 0, s>>>(a, idx, n);
}
