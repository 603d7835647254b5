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
    float4 e[LOG_N];   // 1/c, log c (hi), log c (lo), c
};
__device__ LogTab g_logtab;

constexpr float LN2_H = 0.693147182464599609375f;        // fl(ln 2)
constexpr float LN2_L = -1.904654323148236e-09f;        // ln 2 - LN2_H

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// log of the unevaluated pair (s, corr), s > 0 normal, |corr| <= 2^-24 s, as
// hi + lo with an error of about 1e-13.
__device__ __forceinline__ void ff_log(const float4* __restrict__ tab, float s, float corr, float& hi, float& lo) {
    const int bits = __float_as_int(s);
    // exponent as a float: 2^23 + biased exponent, minus (2^23 + 127)
    const float fe = __fsub_rn(__int_as_float((bits >> 23) | 0x4b000000), 8388735.0f);
    const int i = (bits >> (23 - LOG_BITS)) & (LOG_N - 1);
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);    // [1, 2)
    const float4 t = tab[i];                                             // 1/c, log c (hi, lo), c
    const float u = __fsub_rn(m, t.w);                                   // exact (Sterbenz)
    const float wh = __fmul_rn(u, t.x);
    const float wl = __fmul_rn(__fmaf_rn(-wh, t.w, u), t.x);            // residual u - wh c is exact
    // log(1 + w) - w = -w^2/2 + w^3/3 - w^4/4  (|w| < 2^-10)
    float p = __fmaf_rn(wh, -0.25f, 0.33333334f);
    p = __fmaf_rn(wh, p, -0.5f);
    p = __fmul_rn(__fmul_rn(p, wh), wh);
    const float P = __fmul_rn(fe, LN2_H);
    const float eP = __fmaf_rn(fe, LN2_H, -P);                          // exact product error
    // |P| >= ln 2 > log c whenever E != 0, and P = 0 otherwise: fast two-sum
    const float a = __fadd_rn(P, t.y);
    const float ea = __fsub_rn(t.y, __fsub_rn(a, P));
    float b, eb;
    two_sum(a, wh, b, eb);
    float rs;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(s));             // corr/s is ~2^-24: an approximate 1/s suffices
    float tail = __fadd_rn(__fmaf_rn(-wh, wl, wl), __fmul_rn(corr, rs));
    tail = __fadd_rn(tail, __fmaf_rn(fe, LN2_L, t.z));
    tail = __fadd_rn(tail, p);
    tail = __fadd_rn(tail, __fadd_rn(__fadd_rn(ea, eb), eP));
    hi = b;
    lo = tail;
}

// |x_t - y_s|^2 as a renormalised float-float pair from the split coordinates
// (hi parts on a common dyadic grid, so hi_t - hi_s is exact).
__device__ __forceinline__ void ff_dist2(float thx, float thy, float tlx, float tly, float4 sv, float& s, float& corr) {
    const float a = __fsub_rn(thx, sv.x), b = __fsub_rn(thy, sv.y);
    const float al = __fsub_rn(tlx, sv.z), bl = __fsub_rn(tly, sv.w);
    const float dxh = __fadd_rn(a, al), dyh = __fadd_rn(b, bl);      // |a| >= |al| or a = 0
    const float dxl = __fadd_rn(__fsub_rn(a, dxh), al), dyl = __fadd_rn(__fsub_rn(b, dyh), bl);
    const float p1 = __fmul_rn(dxh, dxh), p2 = __fmul_rn(dyh, dyh);
    const float e1 = __fmaf_rn(dxh, dxh, -p1), e2 = __fmaf_rn(dyh, dyh, -p2);
    const float big = fmaxf(p1, p2), small = fminf(p1, p2);
    const float s0 = __fadd_rn(big, small);
    const float e3 = __fsub_rn(small, __fsub_rn(s0, big));            // fast two-sum (big >= small >= 0)
    float c0 = __fadd_rn(__fadd_rn(e1, e2), e3);
    c0 = __fmaf_rn(2.0f, __fmaf_rn(dxh, dxl, __fmul_rn(dyh, dyl)), c0);
    s = __fadd_rn(s0, c0);                                           // renormalise: |corr| <= 2^-24 s
    corr = __fadd_rn(__fsub_rn(s0, s), c0);
    if (!(s > 1e-30f)) {                                             // coincident points (guarded by callers)
        s = 1e-30f;
        corr = 0.0f;
    }
}

// acc += q * log r^2 in float-float: exact product error and two-sum.
__device__ __forceinline__ void ff_madd(float qh, float ql, float lh, float ll, float& sh, float& sl) {
    const float pr = __fmul_rn(qh, lh);
    const float pe = __fmaf_rn(qh, lh, -pr);
    const float lo_t = __fmaf_rn(qh, ll, __fmaf_rn(ql, lh, pe));
    float ns, ne;
    two_sum(sh, pr, ns, ne);
    sh = ns;
    sl = __fadd_rn(sl, __fadd_rn(ne, lo_t));
}

constexpr int FF_THREADS = 128;
constexpr int FF_TILE = 128;
constexpr int FF_TPT = 2;   // targets per thread: target t and t + FF_THREADS of the block

template <int D, bool CHECK_OWN>
__device__ __forceinline__ void ff_tile(const float4* __restrict__ sxy, const float (*sq)[2 * D],
                                        const float4* __restrict__ stab, int nt, const float* thx, const float* thy,
                                        const float* tlx, const float* tly, const int* own_local,
                                        float (*sh)[D], float (*sl)[D]) {
#pragma unroll 2
    for (int i = 0; i < nt; i++) {
        const float4 sv = sxy[i];
        float qh[D], ql[D];
#pragma unroll
        for (int k = 0; k < D; k++) {
            qh[k] = sq[i][k];
            ql[k] = sq[i][D + k];
        }
#pragma unroll
        for (int r = 0; r < FF_TPT; r++) {
            float s, corr;
            ff_dist2(thx[r], thy[r], tlx[r], tly[r], sv, s, corr);
            if (CHECK_OWN && i == own_local[r]) {                    // own node: log 1 = 0
                s = 1.0f;
                corr = 0.0f;
            }
            float lh, ll;
            ff_log(stab, s, corr, lh, ll);                           // log |x-y|^2 = lh + ll
#pragma unroll
            for (int k = 0; k < D; k++) ff_madd(qh[k], ql[k], lh, ll, sh[r][k], sl[r][k]);
        }
    }
}

template <int D>
__global__ void __launch_bounds__(FF_THREADS) k_far_ff(const float* __restrict__ shi, const float* __restrict__ slo,
                                                       const float* __restrict__ q, int64_t N,
                                                       const float* __restrict__ thi, const float* __restrict__ tlo,
                                                       const int32_t* __restrict__ tnode, int64_t M, int d, int d0,
                                                       double* __restrict__ partial, int splits) {
    __shared__ float4 sxy[FF_TILE];           // hi x, hi y, lo x, lo y
    __shared__ float sq[FF_TILE][2 * D];
    __shared__ float4 stab[LOG_N];
    __shared__ int own_range[2];
    for (int i = threadIdx.x; i < LOG_N; i += FF_THREADS) stab[i] = g_logtab.e[i];
    if (threadIdx.x == 0) {
        own_range[0] = INT32_MAX;
        own_range[1] = -1;
    }
    __syncthreads();
    const int split = blockIdx.y;
    const int64_t per = (N + splits - 1) / splits;
    const int64_t j0 = split * per, j1 = min(N, j0 + per);
    const int64_t tbase = (int64_t)blockIdx.x * (FF_THREADS * FF_TPT) + threadIdx.x;
    float thx[FF_TPT], thy[FF_TPT], tlx[FF_TPT], tly[FF_TPT];
    int64_t own[FF_TPT];
    bool active[FF_TPT];
#pragma unroll
    for (int r = 0; r < FF_TPT; r++) {
        const int64_t t = tbase + r * FF_THREADS;
        active[r] = t < M;
        thx[r] = active[r] ? thi[2 * t] : 0.f;
        thy[r] = active[r] ? thi[2 * t + 1] : 0.f;
        tlx[r] = active[r] ? tlo[2 * t] : 0.f;
        tly[r] = active[r] ? tlo[2 * t + 1] : 0.f;
        own[r] = active[r] ? (int64_t)tnode[t] : -1;
        if (own[r] >= 0) {
            atomicMin(&own_range[0], (int)own[r]);
            atomicMax(&own_range[1], (int)own[r]);
        }
    }
    __syncthreads();
    const int64_t own_lo = own_range[0], own_hi = own_range[1];
    double acc[FF_TPT][D];
#pragma unroll
    for (int r = 0; r < FF_TPT; r++)
#pragma unroll
        for (int k = 0; k < D; k++) acc[r][k] = 0.0;
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
        float sh[FF_TPT][D], sl[FF_TPT][D];
#pragma unroll
        for (int r = 0; r < FF_TPT; r++)
#pragma unroll
            for (int k = 0; k < D; k++) {
                sh[r][k] = 0.f;
                sl[r][k] = 0.f;
            }
        // only a tile that can hold one of this block's own nodes checks indices
        if (own_hi >= base && own_lo < base + nt) {
            int own_local[FF_TPT];
#pragma unroll
            for (int r = 0; r < FF_TPT; r++) own_local[r] = (own[r] >= base && own[r] < base + nt) ? (int)(own[r] - base) : -1;
            ff_tile<D, true>(sxy, sq, stab, nt, thx, thy, tlx, tly, own_local, sh, sl);
        } else {
            ff_tile<D, false>(sxy, sq, stab, nt, thx, thy, tlx, tly, nullptr, sh, sl);
        }
#pragma unroll
        for (int r = 0; r < FF_TPT; r++)
#pragma unroll
            for (int k = 0; k < D; k++) acc[r][k] += (double)sh[r][k] + (double)sl[r][k];
    }
#pragma unroll
    for (int r = 0; r < FF_TPT; r++) {
        const int64_t t = tbase + r * FF_THREADS;
        if (!active[r]) continue;
#pragma unroll
        for (int k = 0; k < D; k++)
            if (d0 + k < d) partial[((int64_t)split * d + d0 + k) * M + t] = acc[r][k] * (0.5 * VP_INV_TWO_PI);
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
        h.e[i] = make_float4((float)(1.0 / c), lh, (float)(L - (double)lh), (float)c);   // c is exact in float
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
    dim3 grid((unsigned)((M + FF_THREADS * FF_TPT - 1) / (FF_THREADS * FF_TPT)), (unsigned)splits);
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
