// Float-float building blocks of the mixed-precision far sum (shared by the
// single-evaluation and the batched kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

// Log table in shared memory: c_i = 1 + (i + 1/2)/512, rc_i = fl(1/c_i),
// log c_i = lh_i + ll_i (two floats).  Error-free transformations below use
// explicit round-to-nearest intrinsics so the compiler cannot contract them.
constexpr int LOG_BITS = 9;
constexpr int LOG_N = 1 << LOG_BITS;
struct LogTab {
    float4 e[LOG_N];   // 1/c, log c (hi), log c (lo), c
};
// One copy per translation unit (no relocatable device code), filled by
// ensure_logtab() from host code of the same unit.
static __device__ LogTab g_logtab;
// The far sum's table: the same c_i and 1/c_i, log c_i split as a multiple of
// 2^-18 (hi) plus the FP32 rest (lo), so that E ln2_h + hi is exact (ff_log_far).
static __device__ LogTab g_logtab_far;

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

// ln 2 = LN2_H18 + LN2_L18 with LN2_H18 = 181704 2^-18 (18 bits): E LN2_H18 is
// exact for |E| <= 63.
constexpr float LN2_H18 = 0.693145751953125f;
constexpr float LN2_L18 = 1.4286068202862268e-06f;

// The far sum's logarithm of (s, corr), |corr| <= 2^-23 s, s in [2^-63, 2^64),
// trimmed to its error budget.  The far sum's relative error is at most
// max_pair |d log r^2| sum_j |q_j| / (4 pi max|u|); on the workloads here
// sum|q| / (4 pi max|u|) is below 1, so a per-pair error of 1e-11 keeps the
// potential an order of magnitude inside a 1e-10 bar.  With
// log s = E ln 2 + log c + log(1 + w), w = (m - c)/c = wh + wl:
//   * E LN2_H18 (exact) + hi(log c) (on the 2^-18 grid) is exact, so
//     hi + wh + E LN2_H18 takes two fast two-sums (hi >= 2^-10 > |wh|, and
//     |E LN2_H18| >= ln2_h > |hi + wh| or E = 0);
//   * E LN2_L18 + lo(log c) in one FMA: rounding at most 2^-24 (63 + 1)
//     2^-19 = 7e-12 (1e-12 for |E| <= 8, r^2 above 2^-8);
//   * log(1 + w) - w = -w^2/2 + w^3/3 (the dropped w^4/4 < 2^-42), and wl
//     without its w wl part (< 2^-44);
//   * corr / s with an approximate reciprocal (relative 2^-22 of 2^-23);
//   * the result not renormalised (|lo| up to 2^-17 |hi|): the float-float
//     products that follow keep 41 bits, 5e-13 of each term.
// The accurate ff_log (error ~1e-13) stays with the correction weights.
__device__ __forceinline__ void ff_log_far(const float4* __restrict__ tab, float s, float corr, float& hi,
                                           float& lo) {
    const int bits = __float_as_int(s);
    const float fe = __fsub_rn(__int_as_float((bits >> 23) | 0x4b000000), 8388735.0f);
    const int i = (bits >> (23 - LOG_BITS)) & (LOG_N - 1);
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);    // [1, 2)
    const float4 t = tab[i];                                             // 1/c, log c (hi, lo), c
    const float u = __fsub_rn(m, t.w);                                   // exact (Sterbenz)
    const float wh = __fmul_rn(u, t.x);
    const float wl = __fmul_rn(__fmaf_rn(-wh, t.w, u), t.x);            // residual u - wh c is exact
    float p = __fmaf_rn(wh, 0.33333334f, -0.5f);
    p = __fmul_rn(__fmul_rn(p, wh), wh);                                 // -w^2/2 + w^3/3
    const float P = __fmul_rn(fe, LN2_H18);                              // exact
    const float s1 = __fadd_rn(t.y, wh);                                 // fast two-sum, t.y >= 2^-10 > |wh|
    const float e1 = __fsub_rn(wh, __fsub_rn(s1, t.y));
    const float b = __fadd_rn(P, s1);                                    // fast two-sum, |P| >= |s1| or P = 0
    const float e2 = __fsub_rn(s1, __fsub_rn(b, P));
    float rs;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(s));
    float tail = __fmaf_rn(corr, rs, wl);
    tail = __fadd_rn(tail, __fmaf_rn(fe, LN2_L18, t.z));
    tail = __fadd_rn(tail, p);
    tail = __fadd_rn(tail, __fadd_rn(e1, e2));
    // left unnormalised: |tail| reaches 2^-17 |b| (the E LN2_L18 term), so
    // the products that follow keep about 41 bits instead of 47 (q ll is
    // rounded to 2^-24 of itself: 2^-41 of q log r^2, or 2^-24 1e-4 |q|
    // where |b| < |tail| < 1e-4), within the per-pair budget
    hi = b;
    lo = tail;
}

// |x_t - y_s|^2 for the far sum: (a + al)^2 + (b + bl)^2 with a, b the exact
// differences of the hi parts and al, bl of the lo parts, as
// s0 + [e1 + e2 + e3 + al (2a + al) + bl (2b + bl)], s0 + e3 = a^2 + b^2
// exactly (a^2 = p1 + e1, b^2 = p2 + e2), renormalised to (s, corr) with
// |corr| <= 2^-24 s.  The cross terms are rounded to 2^-24 of themselves,
// at most 2^-22 |x - y| q, q the grid of the hi parts: a relative error of
// r^2 below 1e-13 for |x - y| > 1e-4 of the box (the other pairs weigh one
// charge each).  GUARD: map coincident points to s = 1e-30.
template <bool GUARD = true>
__device__ __forceinline__ void ff_dist2_far(float thx, float thy, float tlx, float tly, float4 sv, float& s,
                                             float& corr) {
    const float a = __fsub_rn(thx, sv.x), b = __fsub_rn(thy, sv.y);
    const float al = __fsub_rn(tlx, sv.z), bl = __fsub_rn(tly, sv.w);
    const float p1 = __fmul_rn(a, a), p2 = __fmul_rn(b, b);
    const float e1 = __fmaf_rn(a, a, -p1), e2 = __fmaf_rn(b, b, -p2);
    const float big = fmaxf(p1, p2), small = fminf(p1, p2);
    const float s0 = __fadd_rn(big, small);
    const float e3 = __fsub_rn(small, __fsub_rn(s0, big));            // fast two-sum (big >= small >= 0)
    float c0 = __fadd_rn(__fadd_rn(e1, e2), e3);
    c0 = __fmaf_rn(al, __fmaf_rn(2.0f, a, al), c0);
    c0 = __fmaf_rn(bl, __fmaf_rn(2.0f, b, bl), c0);
    s = __fadd_rn(s0, c0);
    corr = __fadd_rn(__fsub_rn(s0, s), c0);
    if (GUARD && !(s > 1e-30f)) {
        s = 1e-30f;
        corr = 0.0f;
    }
}

// |x_t - y_s|^2 as a renormalised float-float pair from the split coordinates
// (hi parts on a common dyadic grid, so hi_t - hi_s is exact).  GUARD: map
// coincident points to s = 1e-30 (callers that cannot meet them skip it).
template <bool GUARD = true>
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
    if (GUARD && !(s > 1e-30f)) {                                    // coincident points (guarded by callers)
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

template <int D, int TPT, bool CHECK_OWN>
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
        for (int r = 0; r < TPT; r++) {
            float s, corr;
            ff_dist2_far(thx[r], thy[r], tlx[r], tly[r], sv, s, corr);
            if (CHECK_OWN && i == own_local[r]) {                    // own node: log 1 = 0
                s = 1.0f;
                corr = 0.0f;
            }
            float lh, ll;
            ff_log_far(stab, s, corr, lh, ll);                       // log |x-y|^2 = lh + ll
#pragma unroll
            for (int k = 0; k < D; k++) ff_madd(qh[k], ql[k], lh, ll, sh[r][k], sl[r][k]);
        }
    }
}

// Shared memory of one far-sum block.
template <int D>
struct FFSmem {
    float4 sxy[FF_TILE];         // source hi x, hi y, lo x, lo y
    float sq[FF_TILE][2 * D];    // source charges hi..., lo...
    float4 stab[LOG_N];          // log table
    int own_range[2];
};

template <int D>
__device__ __forceinline__ void ff_load_table(FFSmem<D>& sm) {
    for (int i = threadIdx.x; i < LOG_N; i += FF_THREADS) sm.stab[i] = g_logtab_far.e[i];
}

// One block of FF_THREADS x TPT targets (tbase + r FF_THREADS, r < TPT)
// against sources [j0, j1): out[(d0 + k) M + t] = (1/4pi) sum_j q_jk log|x_t - y_j|^2,
// tiles of FF_TILE sources flushed into FP64.  Every thread of the block calls it.
template <int D, int TPT>
__device__ __forceinline__ void ff_far_block(FFSmem<D>& sm, const float* __restrict__ shi,
                                             const float* __restrict__ slo, const float* __restrict__ q, int64_t j0,
                                             int64_t j1, const float* __restrict__ thi, const float* __restrict__ tlo,
                                             const int32_t* __restrict__ tnode, int64_t M, int64_t tbase, int d,
                                             int d0, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        sm.own_range[0] = INT32_MAX;
        sm.own_range[1] = -1;
    }
    __syncthreads();
    float thx[TPT], thy[TPT], tlx[TPT], tly[TPT];
    int64_t own[TPT];
    bool active[TPT];
#pragma unroll
    for (int r = 0; r < TPT; r++) {
        const int64_t t = tbase + r * FF_THREADS;
        active[r] = t < M;
        thx[r] = active[r] ? thi[2 * t] : 0.f;
        thy[r] = active[r] ? thi[2 * t + 1] : 0.f;
        tlx[r] = active[r] ? tlo[2 * t] : 0.f;
        tly[r] = active[r] ? tlo[2 * t + 1] : 0.f;
        own[r] = active[r] ? (int64_t)tnode[t] : -1;
        if (own[r] >= 0) {
            atomicMin(&sm.own_range[0], (int)own[r]);
            atomicMax(&sm.own_range[1], (int)own[r]);
        }
    }
    __syncthreads();
    const int64_t own_lo = sm.own_range[0], own_hi = sm.own_range[1];
    double acc[TPT][D];
#pragma unroll
    for (int r = 0; r < TPT; r++)
#pragma unroll
        for (int k = 0; k < D; k++) acc[r][k] = 0.0;
    for (int64_t base = j0; base < j1; base += FF_TILE) {
        const int nt = (int)min((int64_t)FF_TILE, j1 - base);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += FF_THREADS) {
            const int64_t j = base + i;
            sm.sxy[i] = make_float4(shi[2 * j], shi[2 * j + 1], slo[2 * j], slo[2 * j + 1]);
#pragma unroll
            for (int k = 0; k < 2 * D; k++) sm.sq[i][k] = q[j * 2 * D + k];
        }
        __syncthreads();
        float sh[TPT][D], sl[TPT][D];
#pragma unroll
        for (int r = 0; r < TPT; r++)
#pragma unroll
            for (int k = 0; k < D; k++) {
                sh[r][k] = 0.f;
                sl[r][k] = 0.f;
            }
        // only a tile that can hold one of this block's own nodes checks indices
        if (own_hi >= base && own_lo < base + nt) {
            int own_local[TPT];
#pragma unroll
            for (int r = 0; r < TPT; r++) own_local[r] = (own[r] >= base && own[r] < base + nt) ? (int)(own[r] - base) : -1;
            ff_tile<D, TPT, true>(sm.sxy, sm.sq, sm.stab, nt, thx, thy, tlx, tly, own_local, sh, sl);
        } else {
            ff_tile<D, TPT, false>(sm.sxy, sm.sq, sm.stab, nt, thx, thy, tlx, tly, nullptr, sh, sl);
        }
#pragma unroll
        for (int r = 0; r < TPT; r++)
#pragma unroll
            for (int k = 0; k < D; k++) acc[r][k] += (double)sh[r][k] + (double)sl[r][k];
    }
#pragma unroll
    for (int r = 0; r < TPT; r++) {
        const int64_t t = tbase + r * FF_THREADS;
        if (!active[r]) continue;
#pragma unroll
        for (int k = 0; k < D; k++)
            if (d0 + k < d) out[(int64_t)(d0 + k) * M + t] = acc[r][k] * (0.5 * 0.15915494309189533576888376337251);
    }
    __syncthreads();
}

// q_j = W_j f_j as two floats per density: layout [N][2*D] (hi..., lo...);
// with f2out (one density) also f_j itself as a float-float pair, the form
// the streamed correction apply gathers (triangle-major, fd2_stride(nq) pairs
// per triangle).
template <int D>
__global__ void k_prep_q_ff(const double* __restrict__ W, const double* __restrict__ f, int64_t N, int d, int d0,
                            float* __restrict__ q, float2* __restrict__ f2out = nullptr, int nq = 1) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    if (D == 1 && f2out) {
        const double v = f[(int64_t)d0 * N + j];
        const float h = __double2float_rn(v);
        f2out[(j / nq) * fd2_stride(nq) + j % nq] = make_float2(h, __double2float_rn(v - (double)h));
    }
#pragma unroll
    for (int k = 0; k < D; k++) {
        const double v = (d0 + k < d) ? W[j] * f[(int64_t)(d0 + k) * N + j] : 0.0;
        const float h = (float)v;
        q[j * 2 * D + k] = h;
        q[j * 2 * D + D + k] = (float)(v - (double)h);
    }
}

// Fill this unit's g_logtab on the current device (once per device).  Safe to
// call from several host threads; a device is marked loaded only after its
// copy succeeded, and the copy's error is returned.  vp_create calls it (through
// each unit's *_prepare function) so that no evaluation pays for the blocking
// copy or the module load it triggers.
static cudaError_t ensure_logtab() {
    static std::mutex mu;
    static unsigned loaded_mask[4] = {0, 0, 0, 0};   // devices 0..127
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if ((loaded_mask[dev >> 5] >> (dev & 31)) & 1u) return cudaSuccess;
    static LogTab h;
    for (int i = 0; i < LOG_N; i++) {
        const double c = 1.0 + (i + 0.5) / LOG_N;
        // log c in two floats: the split of the double log leaves an error
        // of ~1e-16, far below the 2^-48 the pair can carry
        const double L = std::log(c);
        const float lh = (float)L;
        h.e[i] = make_float4((float)(1.0 / c), lh, (float)(L - (double)lh), (float)c);   // c is exact in float
    }
    e = cudaMemcpyToSymbol(g_logtab, &h, sizeof(h));
    if (e != cudaSuccess) return e;
    for (int i = 0; i < LOG_N; i++) {
        const double c = 1.0 + (i + 0.5) / LOG_N;
        const double L = std::log(c);
        const double hi = std::nearbyint(L * 262144.0) / 262144.0;    // on the 2^-18 grid (>= 2^-10)
        h.e[i] = make_float4((float)(1.0 / c), (float)hi, (float)(L - hi), (float)c);
    }
    e = cudaMemcpyToSymbol(g_logtab_far, &h, sizeof(h));
    if (e == cudaSuccess) loaded_mask[dev >> 5] |= 1u << (dev & 31);
    return e;
}
