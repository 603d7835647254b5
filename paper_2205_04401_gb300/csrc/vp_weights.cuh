// Shared pieces of the correction-weight kernels (k_weights.cu, k_curved.cu):
// warp sizes and stacks, the moment accumulation in the tensor-Legendre basis,
// the reduction of the moments to the nodal weights, the dyadic panel count of
// Section 3.4 and the exact dyadic sub-triangles of Section 3.3.
#pragma once
#include "vp_internal.h"

namespace {


// Stack depth of the warp-wide traversals (FP64 and curved kernels) and
// resident blocks per SM of the float-float self kernel (chosen by timing
// the 16,384-triangle star build: 6 blocks beat the unconstrained register
// allocation by 17%, 5 and 4 were slower).
#ifndef VP_NEAR_STK
#define VP_NEAR_STK 128
#endif
#ifndef VP_SELF_MINB
#define VP_SELF_MINB 4
#endif

constexpr int WARPS = 4;
constexpr int STK = VP_NEAR_STK;   // sub-triangle stack per warp
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

// mu_i -> C_k, lane k of every group of 32 nodes, written to C[p*nq + k]
// (and to C2 when the build keeps a float-float copy).
__device__ __forceinline__ void finish_pair(const WeightsArgs& a, int64_t p, int T, int own, double xx, double xy,
                                            double* m, int lane, const double* rc, const double* lc, double ln2) {
    double v[16];
#pragma unroll
    for (int q = 0; q < VP_NB; q++) v[q] = m[q];
    v[15] = 0.0;
    // index held by this lane after the reduce-scatter: bits 4..1 of the lane
    const double mine = reduce_scatter16(v, lane);
    for (int k0 = 0; k0 < a.nq; k0 += 32) {
        const int k = k0 + lane;
        double s = 0.0;
        const double* Qk = a.Q + (k < a.nq ? k : 0) * VP_NB;
#pragma unroll
        for (int q = 0; q < VP_NB; q++) s = fma(Qk[q], __shfl_sync(0xffffffffu, mine, 2 * q), s);
        if (k < a.nq) {
            if (k != own) {
                const int64_t j = (int64_t)T * a.nq + k;
                const double dx = xx - a.y[2 * j], dy = xy - a.y[2 * j + 1];
                s -= a.W[j] * (vp_logd(dx * dx + dy * dy, rc, lc, ln2) * (0.5 * VP_INV_TWO_PI));
            }
            a.C[p * a.nq + k] = s;
            if (a.C2) {   // float-float copy (h, l = fl(s - h)) for builds that keep one
                const float h = __double2float_rn(s);
                a.C2[p * a.nq + k] = make_float2(h, __double2float_rn(s - (double)h));
            }
        }
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

// N = min{n >= 0 : 2^-n len < dist}.  Scaling by 2^-n is exact, so for
// positive normal len = m1 2^e1 and dist = m2 2^e2 (1 <= m < 2) the test
// compares exponents, then mantissas: N = e1 - e2 + [m1 >= m2], at least 0.
// Integer work on the bit patterns instead of an FP64 loop (GB300's FP64 pipe
// is narrow); other operands take the loop.
__device__ __forceinline__ int dyadic_count(double len, double dist) {
    const long long bl = __double_as_longlong(len), bd = __double_as_longlong(dist);
    const int el = (int)((bl >> 52) & 0x7ff), ed = (int)((bd >> 52) & 0x7ff);
    if (bl > 0 && bd > 0 && el != 0 && ed != 0 && el != 0x7ff && ed != 0x7ff) {
        const long long mask = (1LL << 52) - 1;
        const int n = el - ed + ((bl & mask) >= (bd & mask) ? 1 : 0);
        return n > 0 ? n : 0;
    }
    int n = 0;
    while (ldexp(len, -n) >= dist && n < 1100) n++;
    return n;
}

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

// Children of a split (Section 3.3): (v0,m01,m20), (m01,v1,m12), (m20,m12,v2),
// (m12,m20,m01), numerators at the next scale.
__device__ __forceinline__ void push_children(const SubTri& S, SubTri* stack, int base) {
    const int32_t m01x = S.v[0] + S.v[2], m01y = S.v[1] + S.v[3];
    const int32_t m12x = S.v[2] + S.v[4], m12y = S.v[3] + S.v[5];
    const int32_t m20x = S.v[4] + S.v[0], m20y = S.v[5] + S.v[1];
    const int32_t V0x = 2 * S.v[0], V0y = 2 * S.v[1], V1x = 2 * S.v[2], V1y = 2 * S.v[3];
    const int32_t V2x = 2 * S.v[4], V2y = 2 * S.v[5];
    SubTri ch;
    ch.L = S.L + 1;
    ch.v[0] = V0x; ch.v[1] = V0y; ch.v[2] = m01x; ch.v[3] = m01y; ch.v[4] = m20x; ch.v[5] = m20y;
    stack[base + 0] = ch;
    ch.v[0] = m01x; ch.v[1] = m01y; ch.v[2] = V1x; ch.v[3] = V1y; ch.v[4] = m12x; ch.v[5] = m12y;
    stack[base + 1] = ch;
    ch.v[0] = m20x; ch.v[1] = m20y; ch.v[2] = m12x; ch.v[3] = m12y; ch.v[4] = V2x; ch.v[5] = V2y;
    stack[base + 2] = ch;
    ch.v[0] = m12x; ch.v[1] = m12y; ch.v[2] = m20x; ch.v[3] = m20y; ch.v[4] = m01x; ch.v[5] = m01y;
    stack[base + 3] = ch;
}


}  // namespace
