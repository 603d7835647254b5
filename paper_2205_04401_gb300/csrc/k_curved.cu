// Curved boundary elements (Section 3.1, Eq. for:blend) on the device: nodes
// and weights through the blending map, bounding boxes that hold the curved
// side, point location with the Newton preimage, and the correction weights
// of (target, curved triangle) pairs.
//
// The weights follow the same two schemes as the straight kernels of
// k_weights.cu, carried to the blending map:
//  - near pairs: the subdivision of Section 3.3 in T's reference simplex; the
//    stop test of Section 4.1 on the triangle through the images of the
//    sub-triangle's vertices with J_S = J_T 4^-depth (J_T of the chord); the
//    near rule's nodes mapped through rho with weight w_j 4^-depth |det J_rho|;
//  - self pairs: radius-arclength fans (Section 3.4) in reference coordinates
//    around p = rho^{-1}(x); on the fan over the side P -> Q the point
//    y(r, s) = p + r (P + s (Q - P) - p) and
//      int = int_0^1 int_0^1 [log r + log(|rho(y) - x| / r)] K(y) |det J_rho(y)| r h_r |Q - P| dr ds / 2pi,
//    with the generalized Gaussian rule in r and Gauss-Legendre panels in s,
//    graded toward the parameter s~ of the point of the physical side nearest
//    to x (Newton on the curved side, projection on the straight ones), with
//    the dyadic counts of Section 3.4 from that distance and the physical
//    chord lengths on either side of s~.
// Curved pairs are a small share of all pairs (only boundary triangles are
// curved), so these kernels keep the whole node loop in FP64; the map at the
// quadrature nodes (no decision depends on it) uses Clenshaw sums with fused
// multiply-adds, the decisions the exact-rounding map.
#include "vp_internal.h"
#include "vp_curved.cuh"
#include "vp_weights.cuh"

namespace {

// Nodes and weights of the curved triangles (Theorem 3.1 with |det J_rho|):
// y_j = rho_T(xi_k, eta_k), W_j = w_k det J_rho(xi_k, eta_k).  Runs after the
// straight node kernel; a curved triangle given clockwise is an error (its
// curve would run along the wrong side).
__global__ void k_mesh_nodes_curved(const double* __restrict__ vxy, int64_t nv, const int32_t* __restrict__ tri,
                                    int64_t nt, CurveDev cv, FarRuleDev fr,
                                    const double* __restrict__ tv, double* __restrict__ y, double* __restrict__ W,
                                    int32_t* flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* ax = curve_coef(cv, t);
    if (!ax) return;
    const int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) return;   // flagged by the straight kernel
    if (!(orient_rn(vxy[2 * a], vxy[2 * a + 1], vxy[2 * b], vxy[2 * b + 1], vxy[2 * c], vxy[2 * c + 1]) > 0.0)) {
        atomicOr(flag, VP_DEV_ERR_CURVED_CW);
        return;
    }
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; q++) v[q] = tv[6 * t + q];
    const int nq = fr.nq;
    for (int k = 0; k < nq; k++) {
        const int64_t j = t * nq + k;
        double det;
        geom_map_rn(v, ax, cv.K, fr.x[k], fr.y[k], y + 2 * j, nullptr, &det);
        if (!(det > 0.0)) atomicOr(flag, VP_DEV_ERR_DEGEN);
        W[j] = rn_mul(fr.w[k], det);
    }
}

// Grow the box of a curved triangle by the bound of its deviation from the
// chord triangle: xi (1 - xi - eta) <= 1/4 on the simplex and |T_k| <= 1, so
// the element lies within sum_k |a_k| / 4 of the chord triangle per coordinate.
__global__ void k_curved_bbox(int64_t nt, CurveDev cv, double* __restrict__ bbox) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* ax = curve_coef(cv, t);
    if (!ax) return;
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k <= cv.K; k++) {
        sx += fabs(ax[k]);
        sy += fabs(ax[cv.K + 1 + k]);
    }
    sx = 0.25 * sx * (1.0 + 1e-9) + 1e-300;
    sy = 0.25 * sy * (1.0 + 1e-9) + 1e-300;
    double* b = bbox + 4 * t;
    b[0] -= sx;
    b[1] -= sy;
    b[2] += sx;
    b[3] += sy;
}

// S(x) for targets that are not nodes: the lowest-index element of the cell
// list that holds x (elem_contains_rn: orientation tests, and the Newton
// preimage on curved elements).
__global__ void k_locate_curved(const double* __restrict__ tv, CurveDev cv, const double* __restrict__ txy,
                                const int32_t* __restrict__ order, const int32_t* __restrict__ tcell, int64_t M,
                                GridDev g, int32_t* __restrict__ tself) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int32_t t = order[i];
    if (tself[t] >= 0) return;
    const double xx = txy[2 * t], xy = txy[2 * t + 1];
    const int32_t c = tcell[t];
    const int64_t s0 = g.cell_start[c], s1 = g.cell_start[c + 1];
    for (int64_t k = s0; k < s1; k++) {
        const int32_t T = g.cell_tri[k];
        double v[6];
#pragma unroll
        for (int q = 0; q < 6; q++) v[q] = tv[6 * (int64_t)T + q];
        if (elem_contains_rn(v, curve_coef(cv, T), cv.K, xx, xy)) {
            tself[t] = T;
            return;
        }
    }
}

// Pairs by kind (near / self) and by element (straight / curved):
// counters[0..3] = near straight, self straight, near curved, self curved.
__global__ void k_split_pairs4(const uint8_t* __restrict__ kind, const int32_t* __restrict__ ptri, CurveDev cv,
                               int64_t P, int32_t* __restrict__ near_idx, int32_t* __restrict__ self_idx,
                               int32_t* __restrict__ cnear_idx, int32_t* __restrict__ cself_idx,
                               unsigned long long* counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < P;
    int cls = -1;
    if (valid) cls = (kind[i] == 1 ? 1 : 0) + (cv.cidx[ptri[i]] >= 0 ? 2 : 0);
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    int32_t* outs[4] = {near_idx, self_idx, cnear_idx, cself_idx};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned m = __ballot_sync(0xffffffffu, cls == k);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(&counters[k], (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (cls == k) outs[k][base + __popc(m & lower)] = (int32_t)i;
    }
}

// ------------------------------------------------------- near, curved
__global__ void __launch_bounds__(WARPS * 32) k_weights_near_curved(WeightsArgs a, CurveDev cv,
                                                                    const int32_t* __restrict__ idx, int64_t n) {
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
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; q++) v[q] = a.tv[6 * (int64_t)T + q];
    const double* ax = curve_coef(cv, T);
    const double* dax = curve_dcoef(cv, T);
    const int K = cv.K;
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
    int visited = 0;
    bool overflow = false;
    const unsigned lower = (1u << lane) - 1u;
    while (sp > 0 || nleaf > 0) {
        const bool flush = nleaf > 0 && (sp == 0 || nleaf + 32 > LEAFCAP || nleaf >= 32);
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
                // images of the sub-triangle's vertices under rho
                double ph[6];
#pragma unroll
                for (int i = 0; i < 3; i++)
                    geom_map_rn(v, ax, K, ldexp((double)S.v[2 * i], -S.L), ldexp((double)S.v[2 * i + 1], -S.L),
                                ph + 2 * i, nullptr, nullptr);
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
                    lf.wJ = ldexp(0.5 * VP_INV_TWO_PI, -2 * S.L);   // 4^-depth / 4pi; det J_rho per node
                    leaves[nleaf + __popc(lm & lower)] = lf;
                } else {
                    push_children(S, stack, sp + 4 * __popc(sm & lower));
                }
            }
            nleaf += __popc(lm);
            sp += 4 * __popc(sm);
            __syncwarp();
        } else {
            const int combos = nleaf * VP_NNEAR;
            for (int i = lane; i < combos; i += 32) {
                const int li = i / VP_NNEAR, j = i - li * VP_NNEAR;
                const LeafMap& lf = leaves[li];
                const double zx = nx[j], zy = ny[j];
                const double xi = fma(zy, lf.e2x, fma(zx, lf.e1x, lf.a0x));
                const double eta = fma(zy, lf.e2y, fma(zx, lf.e1y, lf.a0y));
                double y[2], det;
                geom_map_fast(v, ax, dax, K, xi, eta, y, &det);
                const double dx = xx - y[0], dy = xy - y[1];
                const double g = vp_logd(dx * dx + dy * dy, lt.rc, lt.lc, ln2) * (nw[j] * lf.wJ * det);
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

// ------------------------------------------------------- self, curved
// |rho(side(s)) - x|^2 with side(s) = P_r + s d_r in reference coordinates;
// F receives rho(side(s)).
__device__ __forceinline__ double side_dist2_rn(const double* v, const double* ax, int K, double prx, double pry,
                                                double drx, double dry, double s, double xx, double xy, double* F) {
    double yp[2];
    geom_map_rn(v, ax, K, rn_add(prx, rn_mul(s, drx)), rn_add(pry, rn_mul(s, dry)), yp, nullptr, nullptr);
    if (F) {
        F[0] = yp[0];
        F[1] = yp[1];
    }
    const double dx = rn_sub(yp[0], xx), dy = rn_sub(yp[1], xy);
    return rn_add(rn_mul(dx, dx), rn_mul(dy, dy));
}

__global__ void __launch_bounds__(WARPS * 32) k_weights_self_curved(WeightsArgs a, CurveDev cv,
                                                                    const int32_t* __restrict__ idx, int64_t n) {
    __shared__ LogSmem lt;
    load_logtab(a.tab, lt);
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (w >= n) return;
    const double ln2 = a.tab->ln2;
    const int64_t p = idx[w];
    const int T = a.ptri[p], t = a.ptgt[p];
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; q++) v[q] = a.tv[6 * (int64_t)T + q];
    const double* ax = curve_coef(cv, T);
    const double* dax = curve_dcoef(cv, T);
    const int K = cv.K;
    const double xx = a.txy[2 * t], xy = a.txy[2 * t + 1];
    const int own = own_index(a, t, T);
    double pxi, peta;
    geom_inverse_rn(v, ax, K, xx, xy, &pxi, &peta);
    // this lane's Gauss-Legendre node (lane / 2) and four radial nodes
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
        // reference side e: (0,0)->(1,0), (1,0)->(0,1), (0,1)->(0,0)
        const double prx = e == 1 ? 1.0 : 0.0, pry = e == 2 ? 1.0 : 0.0;
        const double qrx = e == 0 ? 1.0 : 0.0, qry = e == 1 ? 1.0 : 0.0;
        const double drx = rn_sub(qrx, prx), dry = rn_sub(qry, pry);
        const double Lr = rn_sqrt(rn_add(rn_mul(drx, drx), rn_mul(dry, dry)));
        const double hr = rn_div(fabs(rn_sub(rn_mul(drx, rn_sub(peta, pry)), rn_mul(dry, rn_sub(pxi, prx)))), Lr);
        if (hr == 0.0) continue;
        double Pp[2], Qp[2];
        geom_map_rn(v, ax, K, prx, pry, Pp, nullptr, nullptr);
        geom_map_rn(v, ax, K, qrx, qry, Qp, nullptr, nullptr);
        // foot point: projection on the chord, then Newton on d/ds |side(s) - x|^2
        const double cx = rn_sub(Qp[0], Pp[0]), cy = rn_sub(Qp[1], Pp[1]);
        double s = rn_div(rn_add(rn_mul(rn_sub(xx, Pp[0]), cx), rn_mul(rn_sub(xy, Pp[1]), cy)),
                          rn_add(rn_mul(cx, cx), rn_mul(cy, cy)));
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
        if (e == 0 && ax) {
            for (int it = 0; it < 30; it++) {
                const double h = 1e-6;
                const double f0 = side_dist2_rn(v, ax, K, prx, pry, drx, dry, s, xx, xy, nullptr);
                const double fp = side_dist2_rn(v, ax, K, prx, pry, drx, dry, rn_add(s, h), xx, xy, nullptr);
                const double fm = side_dist2_rn(v, ax, K, prx, pry, drx, dry, rn_sub(s, h), xx, xy, nullptr);
                const double d1 = rn_div(rn_sub(fp, fm), rn_mul(2.0, h));
                const double d2 = rn_div(rn_add(rn_sub(fp, rn_mul(2.0, f0)), fm), rn_mul(h, h));
                if (!(d2 > 0.0)) break;
                const double step = rn_div(d1, d2);
                double sn = rn_sub(s, step);
                if (sn < 0.0) sn = 0.0;
                if (sn > 1.0) sn = 1.0;
                if (fabs(rn_sub(sn, s)) < 1e-15) {
                    s = sn;
                    break;
                }
                s = sn;
            }
        }
        double F[2];
        const double delta = rn_sqrt(side_dist2_rn(v, ax, K, prx, pry, drx, dry, s, xx, xy, F));
        const double l0x = rn_sub(F[0], Pp[0]), l0y = rn_sub(F[1], Pp[1]);
        const double l1x = rn_sub(Qp[0], F[0]), l1y = rn_sub(Qp[1], F[1]);
        const double len0 = rn_sqrt(rn_add(rn_mul(l0x, l0x), rn_mul(l0y, l0y)));
        const double len1 = rn_sqrt(rn_add(rn_mul(l1x, l1x), rn_mul(l1y, l1y)));
        for (int side = 0; side < 2; side++) {
            if (side == 0 ? !(s > 0.0) : !(s < 1.0)) continue;
            const int Nd = dyadic_count(side == 0 ? len0 : len1, delta);
            // panel boundaries in the side parameter: b_0 = end, b_i = end -/+
            // (1 - 2^-i) (length in parameter), b_{Nd+1} = s~
            double b0 = side == 0 ? 0.0 : 1.0;
            for (int i = 0; i <= Nd; i++) {
                double b1;
                if (i == Nd) b1 = s;
                else {
                    const double fr = rn_sub(1.0, ldexp(1.0, -(i + 1)));
                    b1 = side == 0 ? rn_mul(fr, s) : rn_sub(1.0, rn_mul(fr, rn_sub(1.0, s)));
                }
                panels++;
                const double su = b0 + (b1 - b0) * lxg;
                const double ws = fabs((b1 - b0) * lwg) * Lr * hr;
                const double gx = prx + su * drx - pxi, gy = pry + su * dry - peta;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const double r = gr[q];
                    const double yxi = fma(r, gx, pxi), yeta = fma(r, gy, peta);
                    double y[2], det;
                    geom_map_fast(v, ax, dax, K, yxi, yeta, y, &det);
                    const double dx = y[0] - xx, dy = y[1] - xy;
                    // log r + log(|rho(y) - x| / r), the second term smooth in r
                    const double lg = glr[q] + 0.5 * vp_logd((dx * dx + dy * dy) / (r * r), lt.rc, lt.lc, ln2);
                    accumulate(m, lg * ws * gwl[q] * det, yxi, yeta);
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

}  // namespace

void launch_mesh_nodes_curved(const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, CurveDev cv,
                              FarRuleDev fr, const double* tv, double* y, double* W, int32_t* flag, cudaStream_t s) {
    if (nt > 0)
        k_mesh_nodes_curved<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(vxy, nv, tri, nt, cv, fr, tv, y, W, flag);
}

void launch_curved_bbox(int64_t nt, CurveDev cv, double* bbox, cudaStream_t s) {
    if (nt > 0) k_curved_bbox<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(nt, cv, bbox);
}

void launch_locate_curved(const double* tv, CurveDev cv, const double* txy, const int32_t* order,
                          const int32_t* tcell, int64_t M, GridDev g, int32_t* tself, cudaStream_t s) {
    if (M > 0) k_locate_curved<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(tv, cv, txy, order, tcell, M, g, tself);
}

void launch_split_pairs4(const uint8_t* pkind, const int32_t* ptri, CurveDev cv, int64_t P, int32_t* near_idx,
                         int32_t* self_idx, int32_t* cnear_idx, int32_t* cself_idx, unsigned long long* counters,
                         cudaStream_t s) {
    cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s);
    if (P > 0)
        k_split_pairs4<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(pkind, ptri, cv, P, near_idx, self_idx, cnear_idx,
                                                                   cself_idx, counters);
}

void launch_weights_curved(const WeightsArgs& a, CurveDev cv, const int32_t* self_idx, int64_t n_self,
                           const int32_t* near_idx, int64_t n_near, cudaStream_t s, vp_ctx* ctx) {
    const unsigned gs = (unsigned)((n_self + WARPS - 1) / WARPS), gn = (unsigned)((n_near + WARPS - 1) / WARPS);
    PROF(ctx, ST_WEIGHTS_CURVED, s, if (n_self > 0) k_weights_self_curved<<<gs, WARPS * 32, 0, s>>>(a, cv, self_idx, n_self);
         if (n_near > 0) k_weights_near_curved<<<gn, WARPS * 32, 0, s>>>(a, cv, near_idx, n_near));
}
