// Far sum by a fast multipole method (the FMM coupling of Section 3.6, where
// the paper calls a library FMM): u_far(x_t) = sum_{j != own(t)} q_j G(x_t, y_j),
// q_j = W_j f_j, G = log|x - y| / 2pi, over a uniform quadtree of L levels on
// a square holding every node and target.
//
// Expansions (complex FP64, P terms, scaled by the box side r):
//   multipole about c:  phi(z) = a_0 log(z - c) + sum_k a_k (r / (z - c))^k,
//                       a_0 = sum q_i, a_k = -sum q_i ((z_i - c)/r)^k / k;
//   local about c:      phi(z) = sum_l b_l ((z - c)/r)^l;
// with the translations of Greengard and Rokhlin: M2M (child to parent),
// M2L between the well-separated boxes of a level (children of the parent's
// neighbours that are not neighbours; its products in float-float, the
// expansions stored in FP64), L2L (parent to child).  The leaves'
// own and adjacent boxes are summed directly (P2P) in the float-float
// arithmetic of the direct far sum, skipping the target's own node.  With
// one box of separation the translation error of a point source at the
// nearest corner of a well-separated box is 2.7e-13 at P = 32 and 4e-16 at
// P = 40 (about 1e-14 at the default P = 36) relative to its own value.
//
// Everything is deterministic: nodes and targets are binned into leaves and
// sorted by index inside each leaf, and every sum runs in a fixed order.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "vp_internal.h"
#include "vp_f2.cuh"
#include "vp_ff.cuh"

#ifndef VP_FMM_P
#define VP_FMM_P 36
#endif

namespace {

constexpr int FP = VP_FMM_P;     // expansion order
constexpr int NC = FP + 1;       // coefficients per expansion
constexpr int FT = 64;           // threads per expansion block (>= NC)
static_assert(NC <= FT, "expansion order too high for the block size");

struct cd {
    double x, y;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }
// acc + a b
__device__ __forceinline__ cd cfma(cd a, cd b, cd acc) {
    return {fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y))};
}

// Geometry of the tree on the device.
struct FmmGeo {
    double ox, oy, side;   // root square: lower-left corner and side
    int L;                 // leaf level
    const int64_t* lvl_off;  // [L + 2] first box of each level in the concatenated arrays
};

__device__ __forceinline__ int64_t lvl_off(const FmmGeo& g, int l) { return g.lvl_off[l]; }
__device__ __forceinline__ cd box_center(const FmmGeo& g, int l, int ix, int iy) {
    const double s = ldexp(g.side, -l);
    return {g.ox + (ix + 0.5) * s, g.oy + (iy + 0.5) * s};
}
__device__ __forceinline__ int leaf_coord(double v, double o, double s, int n) {
    const double c = floor((v - o) / s);
    if (!(c >= 0.0)) return 0;
    if (c >= (double)(n - 1)) return n - 1;
    return (int)c;
}

// ------------------------------------------------------------ binning
__global__ void k_fmm_leaf(const double* __restrict__ xy, int64_t n, FmmGeo g, int32_t* __restrict__ leaf,
                           int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nb = 1 << g.L;
    const double s = ldexp(g.side, -g.L);
    const int ix = leaf_coord(xy[2 * i], g.ox, s, nb), iy = leaf_coord(xy[2 * i + 1], g.oy, s, nb);
    const int b = iy * nb + ix;
    leaf[i] = b;
    atomicAdd(&cnt[b], 1);
}

__global__ void k_fmm_scatter(const int32_t* __restrict__ leaf, int64_t n, int64_t* cursor, int32_t* __restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long p = atomicAdd((unsigned long long*)&cursor[leaf[i]], 1ull);
    perm[p] = (int32_t)i;
}

// counts of level l from level l + 1 (sum of the four children)
__global__ void k_fmm_count_up(int l, FmmGeo g, int32_t* cnt_all) {
    const int nb = 1 << l;
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)nb * nb) return;
    const int ix = (int)(b % nb), iy = (int)(b / nb);
    const int32_t* child = cnt_all + lvl_off(g, l + 1);
    const int nc = nb * 2;
    int32_t s = 0;
    for (int c = 0; c < 4; c++) s += child[(2 * iy + (c >> 1)) * nc + 2 * ix + (c & 1)];
    cnt_all[lvl_off(g, l) + b] = s;
}

// sorted sources: float-float coordinates, and the sorted position of each
// node (for the own-node test of node targets)
__global__ void k_fmm_sort_src(const int32_t* __restrict__ perm, int64_t n, FFCoords src, float4* __restrict__ sxy,
                               int32_t* __restrict__ spos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t j = perm[i];
    sxy[i] = make_float4(src.hi[2 * j], src.hi[2 * j + 1], src.lo[2 * j], src.lo[2 * j + 1]);
    spos[j] = (int32_t)i;
}

// ------------------------------------------------------------ charges
// q_j = W_j f_j in sorted order: FP64 for the expansions, float-float
// (hi, lo) for the direct part.
__global__ void k_fmm_charges(const int32_t* __restrict__ perm, int64_t n, const double* __restrict__ W,
                              const double* __restrict__ f, int d, double* __restrict__ q, float2* __restrict__ q2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t j = perm[i];
    for (int k = 0; k < d; k++) {
        const double v = W[j] * f[(int64_t)k * n + j];
        q[(int64_t)k * n + i] = v;
        const float h = __double2float_rn(v);
        q2[(int64_t)k * n + i] = make_float2(h, __double2float_rn(v - (double)h));
    }
}

// ------------------------------------------------------------ P2M
// One block per (leaf, density): nodes in chunks of CH; thread j < CH forms
// the terms -q_j z_j^k / k of its node in float-float complex arithmetic
// (36 complex products per node would occupy the FP64 pipe), thread k sums
// column k of the chunk in node order in float-float and adds it into FP64.
constexpr int CH = 64;
__constant__ float2 c_inv2[NC];   // 1/k, float-float

__device__ __forceinline__ void c2_mul(f2 ar, f2 ai, f2 br, f2 bi, f2& cr, f2& ci) {
    cr = f2_add(f2_mul(ar, br), f2_neg(f2_mul(ai, bi)));
    ci = f2_add(f2_mul(ar, bi), f2_mul(ai, br));
}

__global__ void __launch_bounds__(FT) k_fmm_p2m(FmmGeo g, const int64_t* __restrict__ start,
                                                const int32_t* __restrict__ perm, const double* __restrict__ yxy,
                                                const float2* __restrict__ q2, int64_t N, cd* __restrict__ M) {
    __shared__ float4 T[CH][NC + 1];
    const int64_t b = blockIdx.x;
    const int dd = blockIdx.y;
    const int64_t s0 = start[b], s1 = start[b + 1];
    const int nb = 1 << g.L;
    cd* out = M + ((int64_t)dd * g.lvl_off[g.L + 1] + lvl_off(g, g.L) + b) * NC;
    const int tid = threadIdx.x;
    if (s1 == s0) {
        if (tid < NC) out[tid] = {0.0, 0.0};
        return;
    }
    const double r = ldexp(g.side, -g.L);
    const cd c = box_center(g, g.L, (int)(b % nb), (int)(b / nb));
    double accx = 0.0, accy = 0.0;
    for (int64_t c0 = s0; c0 < s1; c0 += CH) {
        const int64_t i = c0 + tid;
        if (tid < CH && i < s1) {
            const int32_t j = perm[i];
            const float2 qv = q2[(int64_t)dd * N + i];
            const f2 q = {qv.x, qv.y};
            const f2 zr = f2_from_d((yxy[2 * j] - c.x) / r), zi = f2_from_d((yxy[2 * j + 1] - c.y) / r);
            T[tid][0] = make_float4(q.h, q.l, 0.f, 0.f);
            f2 kr = {1.f, 0.f}, ki = {0.f, 0.f};
            const f2 nq = f2_neg(q);
            for (int k = 1; k <= FP; k++) {
                c2_mul(kr, ki, zr, zi, kr, ki);
                const float2 iv = c_inv2[k];
                const f2 sc = f2_mul(nq, {iv.x, iv.y});
                const f2 tr = f2_mul(kr, sc), ti = f2_mul(ki, sc);
                T[tid][k] = make_float4(tr.h, tr.l, ti.h, ti.l);
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)CH, s1 - c0);
        if (tid < NC) {
            f2 sr = {0.f, 0.f}, si = {0.f, 0.f};
            for (int jj = 0; jj < cnt; jj++) {
                const float4 t = T[jj][tid];
                sr = f2_add(sr, {t.x, t.y});
                si = f2_add(si, {t.z, t.w});
            }
            accx += f2_to_d(sr);
            accy += f2_to_d(si);
        }
        __syncthreads();
    }
    if (tid < NC) out[tid] = {accx, accy};
}

// ------------------------------------------------------------ M2M
// parent at level l from its four children at level l + 1:
//   b_0 = sum a_0,  b_l = sum_c [-a_0 w^l / l + sum_{k=1..l} a_k 2^-k w^(l-k) C(l-1, k-1)],
// w = (child centre - parent centre) / r_parent = (+-1 +- i) / 4.
__global__ void __launch_bounds__(FT) k_fmm_m2m(int l, FmmGeo g, const int32_t* __restrict__ cnt_all,
                                                const double* __restrict__ binom, const cd* __restrict__ wpow,
                                                cd* __restrict__ M) {
    __shared__ cd A[4][NC];
    const int nb = 1 << l;
    const int64_t b = blockIdx.x;
    const int dd = blockIdx.y;
    const int ix = (int)(b % nb), iy = (int)(b / nb);
    const int64_t tot = g.lvl_off[g.L + 1];
    cd* out = M + ((int64_t)dd * tot + lvl_off(g, l) + b) * NC;
    const int tid = threadIdx.x;
    if (cnt_all[lvl_off(g, l) + b] == 0) {
        if (tid < NC) out[tid] = {0.0, 0.0};
        return;
    }
    const int nc = 2 * nb;
    for (int c = 0; c < 4; c++) {
        const int64_t cb = (int64_t)(2 * iy + (c >> 1)) * nc + 2 * ix + (c & 1);
        if (tid < NC) A[c][tid] = M[((int64_t)dd * tot + lvl_off(g, l + 1) + cb) * NC + tid];
    }
    __syncthreads();
    if (tid >= NC) return;
    const int L1 = tid;
    cd acc = {0.0, 0.0};
    for (int c = 0; c < 4; c++) {
        const cd* wp = wpow + c * (2 * NC);   // w_c^n, n = 0..2P+1
        if (L1 == 0) {
            acc = cadd(acc, A[c][0]);
            continue;
        }
        acc = cadd(acc, cscale(wp[L1], -A[c][0].x / L1));      // a_0 is real
        double half = 1.0;
        for (int k = 1; k <= L1; k++) {
            half *= 0.5;
            acc = cfma(A[c][k], cscale(wp[L1 - k], half * binom[(L1 - 1) * (2 * NC) + (k - 1)]), acc);
        }
    }
    out[tid] = acc;
}

// ------------------------------------------------------------ M2L
// b_l += sum_k T_o[k][l] a_k over the well-separated boxes (offset o), with
//   T_o[0][0] = log|v|,  T_o[k][0] = (-1)^k v^-k,
//   T_o[0][l] = -v^-l / l,  T_o[k][l] = (-1)^k C(l+k-1, k-1) v^-(l+k)   (k, l >= 1),
// v = (source centre - target centre) / r, and b_0 += a_0 log r; the
// matrices (level independent with scaled expansions) are built on the host.
// One block per (target box, density) over the boxes of every level 2..L.
// Multipoles as float-float complex values (re h, re l, im h, im l) for the
// M2L products.
__global__ void k_fmm_m_f2(const cd* __restrict__ M, int64_t n, float4* __restrict__ M2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const f2 re = f2_from_d(M[i].x), im = f2_from_d(M[i].y);
    M2[i] = make_float4(re.h, re.l, im.h, im.l);
}

// The products run in float-float (the FP64 pipe would bound them at 4 DFMA
// per complex multiply-add; the FP32 pipe does the float-float ones about five
// times faster): each source box's 37-term sum is accumulated in float-float,
// renormalised after every term, and added into FP64; the local expansion is
// stored in FP64.
__global__ void __launch_bounds__(FT) k_fmm_m2l(FmmGeo g, const int32_t* __restrict__ cnt_src,
                                                const int32_t* __restrict__ cnt_tgt, const float4* __restrict__ T2,
                                                const float4* __restrict__ M2, cd* __restrict__ Lc) {
    __shared__ float4 A[NC];
    const int64_t gb = blockIdx.x + g.lvl_off[2];   // global box index (levels >= 2)
    const int dd = blockIdx.y;
    int l = 2;
    while (l < g.L && gb >= g.lvl_off[l + 1]) l++;
    const int64_t b = gb - g.lvl_off[l];
    const int nb = 1 << l;
    const int ix = (int)(b % nb), iy = (int)(b / nb);
    const int64_t tot = g.lvl_off[g.L + 1];
    const int tid = threadIdx.x;
    double accx = 0.0, accy = 0.0;
    if (cnt_tgt[gb] > 0) {
        const f2 logr = f2_from_d(log(ldexp(g.side, -l)));
        const int px = ix >> 1, py = iy >> 1;
        for (int cy = 2 * (py - 1); cy <= 2 * (py + 1) + 1; cy++) {
            if (cy < 0 || cy >= nb) continue;
            for (int cx = 2 * (px - 1); cx <= 2 * (px + 1) + 1; cx++) {
                if (cx < 0 || cx >= nb) continue;
                const int dx = cx - ix, dy = cy - iy;
                if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;   // neighbours: not well separated
                const int64_t sb = (int64_t)cy * nb + cx;
                if (cnt_src[g.lvl_off[l] + sb] == 0) continue;
                __syncthreads();
                if (tid < NC) A[tid] = M2[((int64_t)dd * tot + g.lvl_off[l] + sb) * NC + tid];
                __syncthreads();
                if (tid < NC) {
                    const float4* To = T2 + (int64_t)((dy + 3) * 7 + (dx + 3)) * NC * NC + tid;   // column tid, k-major
                    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;   // re, im
                    if (tid == 0) f2_acc(ah, al, {A[0].x, A[0].y}, logr);
#pragma unroll 4
                    for (int k = 0; k <= FP; k++) {
                        const float4 a = A[k], t = To[(int64_t)k * NC];
                        f2_acc(ah, al, {a.x, a.y}, {t.x, t.y});
                        f2_acc(ah, al, {-a.z, -a.w}, {t.z, t.w});
                        f2_acc(bh, bl, {a.x, a.y}, {t.z, t.w});
                        f2_acc(bh, bl, {a.z, a.w}, {t.x, t.y});
                        const f2 ra = f2_fast(ah, al), rb = f2_fast(bh, bl);
                        ah = ra.h; al = ra.l; bh = rb.h; bl = rb.l;
                    }
                    accx += (double)ah + (double)al;
                    accy += (double)bh + (double)bl;
                }
            }
        }
    }
    if (tid < NC) Lc[((int64_t)dd * tot + gb) * NC + tid] = {accx, accy};
}

// ------------------------------------------------------------ L2L
// child local += 2^-m sum_{l >= m} C(l, m) w^(l-m) b_l (parent), w = (child
// centre - parent centre) / r_parent.
__global__ void __launch_bounds__(FT) k_fmm_l2l(int l, FmmGeo g, const int32_t* __restrict__ cnt_tgt,
                                                const double* __restrict__ binom, const cd* __restrict__ wpow,
                                                cd* __restrict__ Lc) {
    __shared__ cd B[NC];
    const int nb = 1 << l;                // child level l
    const int64_t b = blockIdx.x;
    const int dd = blockIdx.y;
    const int ix = (int)(b % nb), iy = (int)(b / nb);
    const int64_t tot = g.lvl_off[g.L + 1];
    const int tid = threadIdx.x;
    if (cnt_tgt[g.lvl_off[l] + b] == 0) return;
    const int np = nb >> 1;
    const int64_t pb = (int64_t)(iy >> 1) * np + (ix >> 1);
    if (tid < NC) B[tid] = Lc[((int64_t)dd * tot + g.lvl_off[l - 1] + pb) * NC + tid];
    __syncthreads();
    if (tid >= NC) return;
    const int c = ((iy & 1) << 1) | (ix & 1);
    const cd* wp = wpow + c * (2 * NC);
    const int m = tid;
    cd acc = {0.0, 0.0};
    for (int L1 = m; L1 <= FP; L1++) acc = cfma(B[L1], cscale(wp[L1 - m], binom[(int64_t)L1 * (2 * NC) + m]), acc);
    cd* out = Lc + ((int64_t)dd * tot + g.lvl_off[l] + b) * NC + m;
    *out = cadd(*out, cscale(acc, ldexp(1.0, -m)));
}

// ------------------------------------------------------------ evaluation
// Block per (leaf, run of up to EV_THREADS of its targets): the targets
// against the sources of the 3 x 3 leaves around the leaf, which are three
// contiguous runs of the leaf-sorted sources (one per row of leaves), staged
// through shared memory in tiles; every staged source is read by all threads
// at once.  (A block per leaf would serialise the many targets of the dense
// leaves of a graded mesh on one SM.)  The direct part runs in float-float
// (the own node skipped by its sorted position), flushed into FP64 every 32
// sources of a tile; then each target adds the local expansion of its leaf
// (Horner).  u = P2P / 4pi (log r^2) + Re(L2P) / 2pi.
#ifndef VP_FMM_EV_THREADS
#define VP_FMM_EV_THREADS 128
#endif
constexpr int EV_THREADS = VP_FMM_EV_THREADS;   // targets (and threads) per evaluation block
constexpr int EV_TILE = 256;

__global__ void __launch_bounds__(EV_THREADS) k_fmm_eval(FmmGeo g, const int2* __restrict__ units,
                                                         const int64_t* __restrict__ tstart,
                                                         const int32_t* __restrict__ tperm, int64_t M,
                                                         const double* __restrict__ txy, FFCoords tgt,
                                                         const int32_t* __restrict__ tnode,
                                                         const int32_t* __restrict__ spos,
                                                         const int64_t* __restrict__ sstart,
                                                         const float4* __restrict__ sxy, const float2* __restrict__ q2,
                                                         int64_t N, const cd* __restrict__ Lc, int d,
                                                         double* __restrict__ u) {
    __shared__ float4 stab[LOG_N];
    __shared__ float4 s_xy[EV_TILE];
    __shared__ float2 s_q[EV_TILE];
    const int2 un = units[blockIdx.x];
    const int b = un.x;
    const int64_t t0 = tstart[b] + (int64_t)un.y * EV_THREADS, t1 = min(t0 + EV_THREADS, tstart[b + 1]);
    for (int i = threadIdx.x; i < LOG_N; i += blockDim.x) stab[i] = g_logtab_far.e[i];
    const int nb = 1 << g.L;
    const int ix = b % nb, iy = b / nb;
    const int jx0 = max(ix - 1, 0), jx1 = min(ix + 1, nb - 1);
    int64_t r0[3], r1[3];
    int nr = 0;
    for (int jy = max(iy - 1, 0); jy <= min(iy + 1, nb - 1); jy++) {
        r0[nr] = sstart[(int64_t)jy * nb + jx0];
        r1[nr] = sstart[(int64_t)jy * nb + jx1 + 1];
        nr++;
    }
    const double r = ldexp(g.side, -g.L);
    const cd c = box_center(g, g.L, ix, iy);
    const int64_t tot = g.lvl_off[g.L + 1];
    for (int64_t tb = t0; tb < t1; tb += EV_THREADS) {
        const int64_t ti = tb + threadIdx.x;
        const bool live = ti < t1;
        const int32_t t = live ? tperm[ti] : 0;
        const float thx = tgt.hi[2 * t], thy = tgt.hi[2 * t + 1], tlx = tgt.lo[2 * t], tly = tgt.lo[2 * t + 1];
        const int32_t own = tnode[t];
        const int64_t kown = (live && own >= 0) ? (int64_t)spos[own] : -1;
        for (int dd = 0; dd < d; dd++) {
            double acc = 0.0;
            for (int q = 0; q < nr; q++) {
                for (int64_t k0 = r0[q]; k0 < r1[q]; k0 += EV_TILE) {
                    const int n = (int)min((int64_t)EV_TILE, r1[q] - k0);
                    __syncthreads();
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        s_xy[i] = sxy[k0 + i];
                        s_q[i] = q2[(int64_t)dd * N + k0 + i];
                    }
                    __syncthreads();
                    if (!live) continue;
                    const int kl = (int)(kown - k0);              // own node's slot in this tile, if any
                    for (int i0 = 0; i0 < n; i0 += 32) {
                        const int i1 = min(i0 + 32, n);
                        float sh = 0.f, sl = 0.f;
#pragma unroll 4
                        for (int i = i0; i < i1; i++) {
                            float s2, corr;
                            ff_dist2_far<true>(thx, thy, tlx, tly, s_xy[i], s2, corr);
                            if (i == kl) {                        // own node: log 1 = 0
                                s2 = 1.0f;
                                corr = 0.0f;
                            }
                            float lh, ll;
                            ff_log_far(stab, s2, corr, lh, ll);
                            const float2 qv = s_q[i];
                            ff_madd(qv.x, qv.y, lh, ll, sh, sl);
                        }
                        acc += (double)sh + (double)sl;
                    }
                }
            }
            if (live) {
                const cd z = {(txy[2 * t] - c.x) / r, (txy[2 * t + 1] - c.y) / r};
                const cd* B = Lc + ((int64_t)dd * tot + g.lvl_off[g.L] + b) * NC;
                cd phi = B[FP];
                for (int k = FP - 1; k >= 0; k--) phi = cfma(phi, z, B[k]);
                u[(int64_t)dd * M + t] = acc * VP_INV_FOUR_PI + phi.x * VP_INV_TWO_PI;
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- plan
struct FmmPlan {
    int L = 0;
    double ox = 0, oy = 0, side = 1;
    int64_t nbox_tot = 0;
    std::vector<int64_t> h_lvl_off;
    int64_t* d_lvl_off = nullptr;
    int32_t* d_sleaf = nullptr;     // [N] leaf of each source
    int32_t* d_tleaf = nullptr;     // [M] leaf of each target
    int64_t* d_sstart = nullptr;    // [4^L + 1]
    int32_t* d_sperm = nullptr;     // [N] sources by leaf, ascending inside
    int64_t* d_tstart = nullptr;
    int32_t* d_tperm = nullptr;
    int32_t* d_spos = nullptr;      // [N] sorted position of each node
    int2* d_units = nullptr;        // evaluation blocks: (leaf, run of EV_THREADS targets)
    int64_t n_units = 0;
    int32_t* d_scnt = nullptr;      // [nbox_tot] sources per box, all levels
    int32_t* d_tcnt = nullptr;      // [nbox_tot] targets per box
    float4* d_sxy = nullptr;        // [N] sorted sources, float-float
    double* d_binom = nullptr;      // [2NC][2NC] binomial coefficients
    cd* d_wpow = nullptr;           // [4][2NC] powers of the child offsets
    float4* d_T2 = nullptr;         // [49][NC][NC] M2L matrices of the offsets, k-major, float-float (re h, re l, im h, im l)
};

void fmm_plan_free(FmmPlan* p) {
    if (!p) return;
    void* ps[] = {p->d_lvl_off, p->d_sleaf, p->d_tleaf, p->d_sstart, p->d_sperm, p->d_tstart, p->d_tperm,
                  p->d_spos, p->d_units, p->d_scnt, p->d_tcnt, p->d_sxy, p->d_binom, p->d_wpow, p->d_T2};
    for (void* q : ps)
        if (q) cudaFree(q);
    delete p;
}

static FmmGeo fmm_geo(const FmmPlan* p) {
    FmmGeo g;
    g.ox = p->ox;
    g.oy = p->oy;
    g.side = p->side;
    g.L = p->L;
    g.lvl_off = p->d_lvl_off;
    return g;
}

// Leaf level: the one (3..10) minimising a cost model of the evaluation,
// direct pairs (targets x sources of the 3 x 3 leaves around them) against
// translations (boxes with targets x 27 x NC^2), from host histograms.
static int choose_level(const std::vector<double>& sx, const std::vector<double>& tx, double ox, double oy,
                        double side) {
    int best = 3;
    double best_cost = 1e300;
    for (int L = 3; L <= 10; L++) {
        const int nb = 1 << L;
        const double s = side / nb;
        std::vector<int64_t> cs((size_t)nb * nb, 0), ct((size_t)nb * nb, 0);
        auto cell = [&](double x, double y) {
            int ix = (int)std::floor((x - ox) / s), iy = (int)std::floor((y - oy) / s);
            ix = std::min(std::max(ix, 0), nb - 1);
            iy = std::min(std::max(iy, 0), nb - 1);
            return (int64_t)iy * nb + ix;
        };
        for (size_t i = 0; i < sx.size() / 2; i++) cs[cell(sx[2 * i], sx[2 * i + 1])]++;
        for (size_t i = 0; i < tx.size() / 2; i++) ct[cell(tx[2 * i], tx[2 * i + 1])]++;
        double pairs = 0, boxes = 0;
        for (int iy = 0; iy < nb; iy++)
            for (int ix = 0; ix < nb; ix++) {
                const int64_t nt = ct[(size_t)iy * nb + ix];
                if (!nt) continue;
                boxes += 1;
                int64_t ns = 0;
                for (int jy = std::max(iy - 1, 0); jy <= std::min(iy + 1, nb - 1); jy++)
                    for (int jx = std::max(ix - 1, 0); jx <= std::min(ix + 1, nb - 1); jx++) ns += cs[(size_t)jy * nb + jx];
                pairs += (double)nt * ns;
            }
        // ~100 FP32-pipe instructions per direct pair at 40 T/s against
        // ~8 FP64 operations per translation term at 0.6 T/s (upper levels add ~1/3)
        const double cost = pairs * 100.0 / 40e12 + boxes * (4.0 / 3.0) * 27.0 * NC * NC * 8.0 / 0.6e12;
        if (cost < best_cost) {
            best_cost = cost;
            best = L;
        }
    }
    return best;
}

int fmm_plan_build(vp_ctx* ctx, vp_nf* nf, cudaStream_t s) {
    const vp_mesh* mesh = nf->mesh;
    const int64_t N = mesh->N, M = nf->M;
    FmmPlan* p = new (std::nothrow) FmmPlan();
    if (!p) return VP_ERR_OOM;
    auto fail = [&](int code, const char* msg) {
        fmm_plan_free(p);
        return vp_set_error(ctx, code, msg);
    };
    // host copies of the coordinates for the box and the level choice
    std::vector<double> sx(2 * N), tx(2 * M);
    if (cudaMemcpyAsync(sx.data(), mesh->d_y, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(tx.data(), nf->d_txy, 2 * M * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(VP_ERR_CUDA, "fmm plan: coordinate copy failed");
    double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
    for (int64_t i = 0; i < N; i++) {
        x0 = std::min(x0, sx[2 * i]); x1 = std::max(x1, sx[2 * i]);
        y0 = std::min(y0, sx[2 * i + 1]); y1 = std::max(y1, sx[2 * i + 1]);
    }
    for (int64_t i = 0; i < M; i++) {
        x0 = std::min(x0, tx[2 * i]); x1 = std::max(x1, tx[2 * i]);
        y0 = std::min(y0, tx[2 * i + 1]); y1 = std::max(y1, tx[2 * i + 1]);
    }
    const double side = std::max(x1 - x0, y1 - y0) * (1.0 + 1e-9) + 1e-300;
    p->side = side;
    p->ox = 0.5 * (x0 + x1) - 0.5 * side;
    p->oy = 0.5 * (y0 + y1) - 0.5 * side;
    p->L = choose_level(sx, tx, p->ox, p->oy, side);
    const int L = p->L;
    p->h_lvl_off.assign(L + 2, 0);
    for (int l = 0; l <= L; l++) p->h_lvl_off[l + 1] = p->h_lvl_off[l] + ((int64_t)1 << (2 * l));
    p->nbox_tot = p->h_lvl_off[L + 1];
    const int64_t nleaf = (int64_t)1 << (2 * L);
    // tables: binomials, child-offset powers, M2L offset powers
    std::vector<double> binom((size_t)(2 * NC) * (2 * NC), 0.0);
    for (int n = 0; n < 2 * NC; n++) {
        binom[(size_t)n * 2 * NC] = 1.0;
        for (int k = 1; k <= n; k++)
            binom[(size_t)n * 2 * NC + k] = binom[(size_t)(n - 1) * 2 * NC + k - 1] + (k <= n - 1 ? binom[(size_t)(n - 1) * 2 * NC + k] : 0.0);
    }
    std::vector<cd> wpow((size_t)4 * 2 * NC);
    for (int c = 0; c < 4; c++) {
        const long double wx = ((c & 1) ? 0.25L : -0.25L), wy = ((c >> 1) ? 0.25L : -0.25L);
        long double px = 1.0L, py = 0.0L;
        for (int n = 0; n < 2 * NC; n++) {
            wpow[(size_t)c * 2 * NC + n] = {(double)px, (double)py};
            const long double nx = px * wx - py * wy, ny = px * wy + py * wx;
            px = nx;
            py = ny;
        }
    }
    // M2L matrices T_o[k][l] (long double), offsets (dx, dy) in [-3, 3]^2
    std::vector<cd> Tm((size_t)49 * NC * NC, cd{0.0, 0.0});
    for (int dy = -3; dy <= 3; dy++)
        for (int dx = -3; dx <= 3; dx++) {
            const int o = (dy + 3) * 7 + (dx + 3);
            const long double n2 = (long double)dx * dx + (long double)dy * dy;
            if (n2 < 4.0L) continue;   // neighbours never use a matrix
            const long double ix = dx / n2, iy = -dy / n2;   // 1 / (dx + i dy)
            std::vector<long double> pr(2 * NC), pi(2 * NC);
            pr[0] = 1.0L;
            pi[0] = 0.0L;
            for (int n = 1; n < 2 * NC; n++) {
                pr[n] = pr[n - 1] * ix - pi[n - 1] * iy;
                pi[n] = pr[n - 1] * iy + pi[n - 1] * ix;
            }
            auto put = [&](int k, int l, long double re, long double im) {
                Tm[(size_t)o * NC * NC + (size_t)k * NC + l] = {(double)re, (double)im};
            };
            put(0, 0, 0.5L * std::log(n2), 0.0L);
            for (int k = 1; k <= FP; k++) {
                const long double sg = (k & 1) ? -1.0L : 1.0L;
                put(k, 0, sg * pr[k], sg * pi[k]);
            }
            for (int l = 1; l <= FP; l++) {
                put(0, l, -pr[l] / l, -pi[l] / l);
                for (int k = 1; k <= FP; k++) {
                    const long double sg = (k & 1) ? -1.0L : 1.0L;
                    // C(l + k - 1, k - 1)
                    long double c = 1.0L;
                    for (int i = 1; i <= k - 1; i++) c = c * (l + i) / i;
                    put(k, l, sg * c * pr[l + k], sg * c * pi[l + k]);
                }
            }
        }
    cudaError_t e = cudaSuccess;
    auto al = [&](auto** ptr, size_t count) {
        if (e == cudaSuccess) e = cudaMalloc((void**)ptr, std::max<size_t>(1, count) * sizeof(**ptr));
    };
    al(&p->d_lvl_off, L + 2);
    al(&p->d_sleaf, N);
    al(&p->d_tleaf, M);
    al(&p->d_sstart, nleaf + 1);
    al(&p->d_tstart, nleaf + 1);
    al(&p->d_sperm, N);
    al(&p->d_tperm, M);
    al(&p->d_spos, N);
    al(&p->d_scnt, p->nbox_tot);
    al(&p->d_tcnt, p->nbox_tot);
    al(&p->d_sxy, N);
    al(&p->d_binom, binom.size());
    al(&p->d_wpow, wpow.size());
    al(&p->d_T2, Tm.size());
    int64_t* d_cursor = nullptr;
    al(&d_cursor, nleaf + 1);
    if (e != cudaSuccess) {
        if (d_cursor) cudaFree(d_cursor);
        return fail(VP_ERR_OOM, "fmm plan: device allocation failed");
    }
    cudaMemcpyAsync(p->d_lvl_off, p->h_lvl_off.data(), (L + 2) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_binom, binom.data(), binom.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_wpow, wpow.data(), wpow.size() * sizeof(cd), cudaMemcpyHostToDevice, s);
    std::vector<float4> T2(Tm.size());
    for (size_t i = 0; i < Tm.size(); i++) {
        const float rh = (float)Tm[i].x, ih = (float)Tm[i].y;
        T2[i] = make_float4(rh, (float)(Tm[i].x - (double)rh), ih, (float)(Tm[i].y - (double)ih));
    }
    cudaMemcpy(p->d_T2, T2.data(), T2.size() * sizeof(float4), cudaMemcpyHostToDevice);
    {
        float2 inv[NC];
        inv[0] = make_float2(0.f, 0.f);
        for (int k = 1; k < NC; k++) {
            const double v = 1.0 / k;
            const float h = (float)v;
            inv[k] = make_float2(h, (float)(v - (double)h));
        }
        cudaMemcpyToSymbolAsync(c_inv2, inv, sizeof(inv), 0, cudaMemcpyHostToDevice, s);
    }
    const FmmGeo g = fmm_geo(p);
    int rc = VP_OK;
    // bin, count, scan, scatter, sort inside each leaf (sources, then targets)
    struct Side {
        const double* xy;
        int64_t n;
        int32_t* leaf;
        int64_t* start;
        int32_t* perm;
        int32_t* cnt;
    } sides[2] = {{mesh->d_y, N, p->d_sleaf, p->d_sstart, p->d_sperm, p->d_scnt},
                  {nf->d_txy, M, p->d_tleaf, p->d_tstart, p->d_tperm, p->d_tcnt}};
    for (auto& sd : sides) {
        int32_t* leafcnt = sd.cnt + p->h_lvl_off[L];
        cudaMemsetAsync(sd.cnt, 0, p->nbox_tot * sizeof(int32_t), s);
        k_fmm_leaf<<<(unsigned)((sd.n + 255) / 256), 256, 0, s>>>(sd.xy, sd.n, g, sd.leaf, leafcnt);
        rc = vp_exclusive_scan_i32(ctx, leafcnt, sd.start, nleaf, s);
        if (rc) break;
        cudaMemcpyAsync(d_cursor, sd.start, (nleaf + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        k_fmm_scatter<<<(unsigned)((sd.n + 255) / 256), 256, 0, s>>>(sd.leaf, sd.n, d_cursor, sd.perm);
        // ascending order inside every leaf (deterministic sums)
        int32_t* d_max = (int32_t*)d_cursor;   // reuse: the cursor is no longer needed
        launch_max_i32(leafcnt, nleaf, d_max, s);
        int32_t h_max = 0;
        cudaMemcpyAsync(&h_max, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (h_max > 16384) {
            rc = vp_set_error(ctx, VP_ERR_INVALID_ARG, "fmm plan: a leaf holds more than 16384 points");
            break;
        }
        GridDev gd{};
        gd.cell_start = sd.start;
        gd.cell_tri = sd.perm;
        gd.nx = 1 << L;
        gd.ny = 1 << L;
        cudaMemsetAsync(ctx->d_flag, 0, sizeof(int32_t), s);
        launch_cell_sort(gd, nleaf, std::max(h_max, 1), sd.perm, ctx->d_flag, s);
        for (int l = L - 1; l >= 0; l--) {
            const int64_t nb2 = (int64_t)1 << (2 * l);
            k_fmm_count_up<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(l, g, sd.cnt);
        }
    }
    cudaFree(d_cursor);
    if (rc) {
        fmm_plan_free(p);
        return rc;
    }
    ensure_logtab();
    k_fmm_sort_src<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p->d_sperm, N, nf->src_ff, p->d_sxy, p->d_spos);
    if (cudaGetLastError() != cudaSuccess) return fail(VP_ERR_CUDA, "fmm plan: launch failed");
    int32_t h_flag = 0;
    if (cudaMemcpyAsync(&h_flag, ctx->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(VP_ERR_CUDA, "fmm plan: build failed");
    if (h_flag) return fail(VP_ERR_CUDA, "fmm plan: leaf sort exceeded its capacity");
    // evaluation blocks: every leaf's targets in runs of EV_THREADS, heaviest
    // first (targets x sources of the 3 x 3 leaves), so that the blocks that
    // start last are short and the last wave ends together
    {
        std::vector<int64_t> ts(nleaf + 1), ss(nleaf + 1);
        if (cudaMemcpy(ts.data(), p->d_tstart, (nleaf + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(ss.data(), p->d_sstart, (nleaf + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(VP_ERR_CUDA, "fmm plan: copy failed");
        const int nb = 1 << L;
        std::vector<std::pair<int64_t, int2>> wu;
        for (int64_t b = 0; b < nleaf; b++) {
            const int64_t nt = ts[b + 1] - ts[b];
            if (nt == 0) continue;
            const int ix = (int)(b % nb), iy = (int)(b / nb);
            int64_t src = 0;
            for (int jy = std::max(iy - 1, 0); jy <= std::min(iy + 1, nb - 1); jy++)
                src += ss[(int64_t)jy * nb + std::min(ix + 1, nb - 1) + 1] - ss[(int64_t)jy * nb + std::max(ix - 1, 0)];
            for (int64_t k = 0; k * EV_THREADS < nt; k++)
                wu.push_back({std::min<int64_t>(EV_THREADS, nt - k * EV_THREADS) * src, make_int2((int)b, (int)k)});
        }
        std::stable_sort(wu.begin(), wu.end(), [](const std::pair<int64_t, int2>& x, const std::pair<int64_t, int2>& y) {
            return x.first > y.first;
        });
        std::vector<int2> un;
        un.reserve(wu.size());
        for (const auto& w : wu) un.push_back(w.second);
        p->n_units = (int64_t)un.size();
        if (cudaMalloc(&p->d_units, std::max<size_t>(1, un.size()) * sizeof(int2)) != cudaSuccess)
            return fail(VP_ERR_OOM, "fmm plan: device allocation failed");
        if (!un.empty() &&
            cudaMemcpy(p->d_units, un.data(), un.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(VP_ERR_CUDA, "fmm plan: copy failed");
    }
    nf->fmm = p;
    return VP_OK;
}

size_t fmm_ws_bytes(const vp_nf* nf, int d) {
    if (!nf->fmm) return 0;
    const int64_t N = nf->mesh->N;
    return 3 * ((size_t)d * nf->fmm->nbox_tot * NC * sizeof(cd) + 256) + (size_t)d * N * (sizeof(double) + sizeof(float2)) +
           512;
}

int fmm_far(vp_ctx* ctx, const vp_nf* nf, const double* f, int d, double* u, void* ws, cudaStream_t s) {
    const FmmPlan* p = nf->fmm;
    const vp_mesh* mesh = nf->mesh;
    const int64_t N = mesh->N, M = nf->M;
    const FmmGeo g = fmm_geo(p);
    const int L = p->L;
    char* w = (char*)ws;
    auto take = [&](size_t bytes) {
        char* q = w;
        w += (bytes + 255) & ~(size_t)255;
        return q;
    };
    cd* Mp = (cd*)take((size_t)d * p->nbox_tot * NC * sizeof(cd));
    cd* Lc = (cd*)take((size_t)d * p->nbox_tot * NC * sizeof(cd));
    float4* M2 = (float4*)take((size_t)d * p->nbox_tot * NC * sizeof(float4));
    double* q = (double*)take((size_t)d * N * sizeof(double));
    float2* q2 = (float2*)take((size_t)d * N * sizeof(float2));
    const int64_t nleaf = (int64_t)1 << (2 * L);
    k_fmm_charges<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p->d_sperm, N, mesh->d_W, f, d, q, q2);
    k_fmm_p2m<<<dim3((unsigned)nleaf, (unsigned)d), FT, 0, s>>>(g, p->d_sstart, p->d_sperm, mesh->d_y, q2, N, Mp);
    for (int l = L - 1; l >= 2; l--)
        k_fmm_m2m<<<dim3((unsigned)((int64_t)1 << (2 * l)), (unsigned)d), FT, 0, s>>>(l, g, p->d_scnt, p->d_binom,
                                                                                    p->d_wpow, Mp);
    const int64_t n_m2l = p->nbox_tot - p->h_lvl_off[2];
    if (L >= 2) {
        const int64_t nm = (int64_t)d * p->nbox_tot * NC;
        k_fmm_m_f2<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(Mp, nm, M2);
        k_fmm_m2l<<<dim3((unsigned)n_m2l, (unsigned)d), FT, 0, s>>>(g, p->d_scnt, p->d_tcnt, p->d_T2, M2, Lc);
    }
    for (int l = 3; l <= L; l++)
        k_fmm_l2l<<<dim3((unsigned)((int64_t)1 << (2 * l)), (unsigned)d), FT, 0, s>>>(l, g, p->d_tcnt, p->d_binom,
                                                                                    p->d_wpow, Lc);
    if (p->n_units > 0)
        k_fmm_eval<<<(unsigned)p->n_units, EV_THREADS, 0, s>>>(g, p->d_units, p->d_tstart, p->d_tperm, M, nf->d_txy,
                                                               nf->tgt_ff, nf->d_tnode, p->d_spos, p->d_sstart,
                                                               p->d_sxy, q2, N, Lc, d, u);
    VP_LAUNCH_CHECK(ctx);
    return VP_OK;
}

int fmm_level(const vp_nf* nf) { return nf->fmm ? nf->fmm->L : 0; }
int64_t fmm_boxes(const vp_nf* nf) { return nf->fmm ? nf->fmm->nbox_tot : 0; }

// Loads this unit's log table on the current device (vp_create).
cudaError_t fmm_module_prepare() { return ensure_logtab(); }
