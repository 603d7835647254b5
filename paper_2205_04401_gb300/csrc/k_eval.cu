// Potential evaluation: the far sum over all quadrature nodes as point
// charges q_j = W_j f_j (Section 3.6) and the application of the correction
// weights (subtract-and-add).
//
//   u_far(x_t) = sum_{j != own(t)} q_j G(x_t, y_j),   G = log|x - y| / 2pi
//   u(x_t)     = u_far(x_t) + sum_{(t,T) in lists} sum_k C[t,T,k] f_{T,k}
//
// Two far-sum paths:
//  * FP64: tiled all-pairs sum with the library log().
//  * float-float: coordinates split as hi + lo with hi on a dyadic grid so
//    hi_t - hi_s is exact in FP32; |x - y|^2 carried as an unevaluated FP32
//    pair; log of it by a 128-entry table (log c_i in two floats) and the
//    series of log(1 + w) to w^5 with w = (m - c_i)/c_i in two floats;
//    products and sums with exact FP32 error terms (Dekker/Knuth);
//    each tile of sources is flushed into an FP64 accumulator.
#include <cmath>

#include "vp_internal.h"

namespace {

// ------------------------------------------------------------- FP64 far
constexpr int F64_THREADS = 128;
constexpr int F64_TILE = 128;

template <int D>
__global__ void __launch_bounds__(F64_THREADS) k_far_fp64(const double* __restrict__ y, const double* __restrict__ W,
                                                          int64_t N, const double* __restrict__ f, int d, int d0,
                                                          const double* __restrict__ txy, const int32_t* __restrict__ tnode,
                                                          int64_t M, double* __restrict__ partial, int splits) {
    __shared__ double sx[F64_TILE], sy[F64_TILE], sq[D][F64_TILE];
    const int64_t t = (int64_t)blockIdx.x * F64_THREADS + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t per = (N + splits - 1) / splits;
    const int64_t j0 = split * per, j1 = min(N, j0 + per);
    const bool active = t < M;
    const double xx = active ? txy[2 * t] : 0.0, xy = active ? txy[2 * t + 1] : 0.0;
    const int64_t own = active ? (int64_t)tnode[t] : -1;
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; k++) acc[k] = 0.0;
    for (int64_t base = j0; base < j1; base += F64_TILE) {
        const int nt = (int)min((int64_t)F64_TILE, j1 - base);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += F64_THREADS) {
            const int64_t j = base + i;
            sx[i] = y[2 * j];
            sy[i] = y[2 * j + 1];
#pragma unroll
            for (int k = 0; k < D; k++) sq[k][i] = (d0 + k < d) ? W[j] * f[(int64_t)(d0 + k) * N + j] : 0.0;
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < nt; i++) {
                const double dx = xx - sx[i], dy = xy - sy[i];
                double r2 = dx * dx + dy * dy;
                const bool self = (base + i == own);
                const double lg = self ? 0.0 : log(r2);
#pragma unroll
                for (int k = 0; k < D; k++) acc[k] += sq[k][i] * lg;
            }
        }
    }
    if (active) {
#pragma unroll
        for (int k = 0; k < D; k++)
            if (d0 + k < d) partial[((int64_t)split * d + d0 + k) * M + t] = acc[k] * (0.5 * VP_INV_TWO_PI);
    }
}

// out[i] = sum_s partial[s][i] (fixed order)
__global__ void k_reduce_splits(const double* __restrict__ partial, int splits, int64_t count, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s = 0.0;
    for (int k = 0; k < splits; k++) s += partial[(int64_t)k * count + i];
    out[i] = s;
}

// ------------------------------------------------------- corrections
// Warp per target: lanes run over the flattened (pair, node) entries of the
// target's row; u[k][t] += sum C[e] f[k][T_p nq + node].
__global__ void k_apply_fp64(const int64_t* __restrict__ row, const int32_t* __restrict__ ptri,
                             const double* __restrict__ C, int nq, const double* __restrict__ f, int64_t N, int d,
                             int64_t M, double* __restrict__ u) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    const int64_t e0 = row[t] * nq, e1 = row[t + 1] * nq;
    for (int k = 0; k < d; k++) {
        const double* fk = f + (int64_t)k * N;
        double s = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t p = e / nq;
            const int node = (int)(e - p * nq);
            s += C[e] * fk[(int64_t)ptri[p] * nq + node];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) u[(int64_t)k * M + t] += s;
    }
}

// ------------------------------------------------------ float-float far
// Split FP64 coordinates: v - o = hi + lo, hi = q * round((v - o)/q).
__global__ void k_ff_split(const double* __restrict__ xy, int64_t n, double ox, double oy, double q, float* __restrict__ hi,
                           float* __restrict__ lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const double v = xy[2 * i + c] - (c == 0 ? ox : oy);
        const double h = rint(v / q) * q;
        hi[2 * i + c] = (float)h;
        lo[2 * i + c] = (float)(v - h);
    }
}

// q_j = W_j f_j as two floats per density: layout [N][2*D] (hi..., lo...)
template <int D>
__global__ void k_prep_q_ff(const double* __restrict__ W, const double* __restrict__ f, int64_t N, int d, int d0,
                            float* __restrict__ q) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
#pragma unroll
    for (int k = 0; k < D; k++) {
        const double v = (d0 + k < d) ? W[j] * f[(int64_t)(d0 + k) * N + j] : 0.0;
        const float h = (float)v;
        q[j * 2 * D + k] = h;
        q[j * 2 * D + D + k] = (float)(v - (double)h);
    }
}

// Log table in shared memory: c_i = 1 + (i + 1/2)/512, rc_i = fl(1/c_i),
// log c_i = lh_i + ll_i (two floats).  Error-free transformations below use
// explicit round-to-nearest intrinsics so the compiler cannot contract them.
constexpr int LOG_BITS = 9;
constexpr int LOG_N = 1 << LOG_BITS;
struct LogTab {
    float4 e[LOG_N];   // rc, lh, ll, unused
};
__device__ LogTab g_logtab;

constexpr float LN2_H = 0.693147182464599609375f;        // fl(ln 2)
constexpr float LN2_L = -1.904654323148236e-09f;        // ln 2 - LN2_H

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// log of the unevaluated pair (s, corr), s > 0 normal, |corr| <= 2^-20 s, as
// b + tail with |tail| <~ 2^-19 |b| + 2^-21 and an error of about 1e-13.
__device__ __forceinline__ void ff_log(const float4* __restrict__ tab, float s, float corr, float& hi, float& lo) {
    const int bits = __float_as_int(s);
    const int E = ((bits >> 23) & 0xff) - 127;
    const int i = (bits >> (23 - LOG_BITS)) & (LOG_N - 1);
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);    // [1, 2)
    const float c = __fadd_rn(1.0f, __fmul_rn(__fadd_rn((float)i, 0.5f), 1.0f / LOG_N));
    const float4 t = tab[i];
    const float u = __fsub_rn(m, c);                                     // exact (Sterbenz)
    const float wh = __fmul_rn(u, t.x);
    const float wl = __fmul_rn(__fmaf_rn(-wh, c, u), t.x);              // residual u - wh c is exact
    // log(1 + w) - w = -w^2/2 + w^3/3 - w^4/4  (|w| < 2^-10)
    float p = __fmaf_rn(wh, -0.25f, 0.33333334f);
    p = __fmaf_rn(wh, p, -0.5f);
    p = __fmul_rn(__fmul_rn(p, wh), wh);
    const float fe = (float)E;
    const float P = __fmul_rn(fe, LN2_H);
    const float eP = __fmaf_rn(fe, LN2_H, -P);                          // exact product error
    float a, ea, b, eb;
    two_sum(P, t.y, a, ea);
    two_sum(a, wh, b, eb);
    float tail = __fadd_rn(__fmaf_rn(-wh, wl, wl), __fmul_rn(corr, __frcp_rn(s)));
    tail = __fadd_rn(tail, __fmaf_rn(fe, LN2_L, t.z));
    tail = __fadd_rn(tail, p);
    tail = __fadd_rn(tail, __fadd_rn(__fadd_rn(ea, eb), eP));
    hi = b;
    lo = tail;
}

constexpr int FF_THREADS = 128;
constexpr int FF_TILE = 128;

template <int D>
__global__ void __launch_bounds__(FF_THREADS) k_far_ff(const float* __restrict__ shi, const float* __restrict__ slo,
                                                       const float* __restrict__ q, int64_t N,
                                                       const float* __restrict__ thi, const float* __restrict__ tlo,
                                                       const int32_t* __restrict__ tnode, int64_t M, int d, int d0,
                                                       double* __restrict__ partial, int splits) {
    __shared__ float4 sxy[FF_TILE];           // hi x, hi y, lo x, lo y
    __shared__ float sq[FF_TILE][2 * D];
    __shared__ float4 stab[LOG_N];
    for (int i = threadIdx.x; i < LOG_N; i += FF_THREADS) stab[i] = g_logtab.e[i];
    const int64_t t = (int64_t)blockIdx.x * FF_THREADS + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t per = (N + splits - 1) / splits;
    const int64_t j0 = split * per, j1 = min(N, j0 + per);
    const bool active = t < M;
    const float thx = active ? thi[2 * t] : 0.f, thy = active ? thi[2 * t + 1] : 0.f;
    const float tlx = active ? tlo[2 * t] : 0.f, tly = active ? tlo[2 * t + 1] : 0.f;
    const int64_t own = active ? (int64_t)tnode[t] : -1;
    double acc[D];
#pragma unroll
    for (int k = 0; k < D; k++) acc[k] = 0.0;
    for (int64_t base = j0; base < j1; base += FF_TILE) {
        const int nt = (int)min((int64_t)FF_TILE, j1 - base);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += FF_THREADS) {
            const int64_t j = base + i;
            sxy[i] = make_float4(shi[2 * j], shi[2 * j + 1], slo[2 * j], slo[2 * j + 1]);
#pragma unroll
            for (int k = 0; k < 2 * D; k++) sq[i][k] = q[j * 2 * D + k];
        }
        __syncthreads();
        if (active) {
            float sh[D], sl[D];
#pragma unroll
            for (int k = 0; k < D; k++) { sh[k] = 0.f; sl[k] = 0.f; }
            const int64_t own_local = own - base;
            for (int i = 0; i < nt; i++) {
                const float4 sv = sxy[i];
                // dx = (hi_t - hi_s) + (lo_t - lo_s): the hi difference is exact
                // (same dyadic grid); renormalise to a float-float pair
                const float a = __fsub_rn(thx, sv.x), b = __fsub_rn(thy, sv.y);
                const float al = __fsub_rn(tlx, sv.z), bl = __fsub_rn(tly, sv.w);
                const float dxh = __fadd_rn(a, al), dyh = __fadd_rn(b, bl);    // |a| >= |al| or a = 0
                const float dxl = __fadd_rn(__fsub_rn(a, dxh), al), dyl = __fadd_rn(__fsub_rn(b, dyh), bl);
                // r^2 = dxh^2 + dyh^2 + 2 (dxh dxl + dyh dyl) with exact product errors
                const float p1 = __fmul_rn(dxh, dxh), p2 = __fmul_rn(dyh, dyh);
                const float e1 = __fmaf_rn(dxh, dxh, -p1), e2 = __fmaf_rn(dyh, dyh, -p2);
                const float big = fmaxf(p1, p2), small = fminf(p1, p2);
                float s0 = __fadd_rn(big, small);
                const float e3 = __fsub_rn(small, __fsub_rn(s0, big));  // fast two-sum (big >= small >= 0)
                float c0 = __fadd_rn(__fadd_rn(e1, e2), e3);
                c0 = __fmaf_rn(2.0f, __fmaf_rn(dxh, dxl, __fmul_rn(dyh, dyl)), c0);
                // renormalise (s0, c0) so that |corr| <= 2^-24 s before the logarithm
                float s = __fadd_rn(s0, c0);
                float corr = __fadd_rn(__fsub_rn(s0, s), c0);
                if (!(s > 1e-30f)) { s = 1e-30f; corr = 0.0f; }        // coincident points (guarded by callers)
                if (i == own_local) { s = 1.0f; corr = 0.0f; }         // own node: log 1 = 0
                float lh, ll;
                ff_log(stab, s, corr, lh, ll);                         // log |x-y|^2 = lh + ll
#pragma unroll
                for (int k = 0; k < D; k++) {
                    const float qh = sq[i][k], ql = sq[i][D + k];
                    const float pr = __fmul_rn(qh, lh);
                    const float pe = __fmaf_rn(qh, lh, -pr);
                    const float lo_t = __fmaf_rn(qh, ll, __fmaf_rn(ql, lh, pe));
                    float ns, ne;
                    two_sum(sh[k], pr, ns, ne);
                    sh[k] = ns;
                    sl[k] = __fadd_rn(sl[k], __fadd_rn(ne, lo_t));
                }
            }
#pragma unroll
            for (int k = 0; k < D; k++) acc[k] += (double)sh[k] + (double)sl[k];
        }
    }
    if (active) {
#pragma unroll
        for (int k = 0; k < D; k++)
            if (d0 + k < d) partial[((int64_t)split * d + d0 + k) * M + t] = acc[k] * (0.5 * VP_INV_TWO_PI);
    }
}

int g_logtab_device = -1;

void ensure_logtab() {
    int dev = -1;
    cudaGetDevice(&dev);
    if (g_logtab_device == dev) return;
    static LogTab h;
    for (int i = 0; i < LOG_N; i++) {
        const double c = 1.0 + (i + 0.5) / LOG_N;
        // log c in two floats: the split of the double log leaves an error
        // of ~1e-16, far below the 2^-48 the pair can carry
        const double L = std::log(c);
        const float lh = (float)L;
        h.e[i] = make_float4((float)(1.0 / c), lh, (float)(L - (double)lh), 0.0f);
    }
    cudaMemcpyToSymbol(g_logtab, &h, sizeof(h));
    g_logtab_device = dev;
}

int pick_chunk(int d) { return d >= 8 ? 8 : (d >= 4 ? 4 : (d >= 2 ? 2 : 1)); }

}  // namespace

void launch_far_fp64(const double* y, const double* W, int64_t N, const double* f, int d, const double* txy,
                     const int32_t* tnode, int64_t M, double* partial, int splits, cudaStream_t s) {
    dim3 grid((unsigned)((M + F64_THREADS - 1) / F64_THREADS), (unsigned)splits);
    for (int d0 = 0; d0 < d;) {
        const int D = pick_chunk(d - d0);
        switch (D) {
            case 8: k_far_fp64<8><<<grid, F64_THREADS, 0, s>>>(y, W, N, f, d, d0, txy, tnode, M, partial, splits); break;
            case 4: k_far_fp64<4><<<grid, F64_THREADS, 0, s>>>(y, W, N, f, d, d0, txy, tnode, M, partial, splits); break;
            case 2: k_far_fp64<2><<<grid, F64_THREADS, 0, s>>>(y, W, N, f, d, d0, txy, tnode, M, partial, splits); break;
            default: k_far_fp64<1><<<grid, F64_THREADS, 0, s>>>(y, W, N, f, d, d0, txy, tnode, M, partial, splits); break;
        }
        d0 += D;
    }
}

void launch_far_ff(const FFCoords& src, const double* W, int64_t N, const double* f, int d, const FFCoords& tgt,
                   const int32_t* tnode, int64_t M, double* partial, float* qbuf, int splits, cudaStream_t s) {
    ensure_logtab();
    dim3 grid((unsigned)((M + FF_THREADS - 1) / FF_THREADS), (unsigned)splits);
    const unsigned pb = (unsigned)((N + 255) / 256);
    for (int d0 = 0; d0 < d;) {
        const int D = pick_chunk(d - d0);
        switch (D) {
            case 8:
                k_prep_q_ff<8><<<pb, 256, 0, s>>>(W, f, N, d, d0, qbuf);
                k_far_ff<8><<<grid, FF_THREADS, 0, s>>>(src.hi, src.lo, qbuf, N, tgt.hi, tgt.lo, tnode, M, d, d0, partial, splits);
                break;
            case 4:
                k_prep_q_ff<4><<<pb, 256, 0, s>>>(W, f, N, d, d0, qbuf);
                k_far_ff<4><<<grid, FF_THREADS, 0, s>>>(src.hi, src.lo, qbuf, N, tgt.hi, tgt.lo, tnode, M, d, d0, partial, splits);
                break;
            case 2:
                k_prep_q_ff<2><<<pb, 256, 0, s>>>(W, f, N, d, d0, qbuf);
                k_far_ff<2><<<grid, FF_THREADS, 0, s>>>(src.hi, src.lo, qbuf, N, tgt.hi, tgt.lo, tnode, M, d, d0, partial, splits);
                break;
            default:
                k_prep_q_ff<1><<<pb, 256, 0, s>>>(W, f, N, d, d0, qbuf);
                k_far_ff<1><<<grid, FF_THREADS, 0, s>>>(src.hi, src.lo, qbuf, N, tgt.hi, tgt.lo, tnode, M, d, d0, partial, splits);
                break;
        }
        d0 += D;
    }
}

void launch_reduce_splits(const double* partial, int splits, int64_t count, double* out, cudaStream_t s) {
    if (count > 0) k_reduce_splits<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(partial, splits, count, out);
}

void launch_apply_fp64(const int64_t* row, const int32_t* ptri, const double* C, int nq, const double* f, int64_t N,
                       int d, int64_t M, double* u, cudaStream_t s) {
    if (M > 0) k_apply_fp64<<<(unsigned)((M * 32 + 255) / 256), 256, 0, s>>>(row, ptri, C, nq, f, N, d, M, u);
}

void launch_ff_split(const double* xy, int64_t n, double ox, double oy, double q, FFCoords out, cudaStream_t s) {
    if (n > 0) k_ff_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, n, ox, oy, q, out.hi, out.lo);
}
