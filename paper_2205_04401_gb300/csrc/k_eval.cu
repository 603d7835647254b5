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
#include "vp_ff.cuh"

namespace {

int pick_chunk(int d) { return d >= 8 ? 8 : (d >= 4 ? 4 : (d >= 2 ? 2 : 1)); }

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
// Few densities: warp per target; lanes run over the flattened (pair, node)
// entries of the target's row, each entry's weight read once for D densities;
// u[d0 + k][t] += sum C[e] f[d0 + k][T_p nq + node].  Eight entries per lane
// are in flight (predicated, no tail loop) and u[t] is fetched before the
// row, so a warp has up to 16 independent loads outstanding.
// NQ = 0: nodes per triangle given at run time (generated far rules).
template <int NQ, int D>
__global__ void __launch_bounds__(256) k_apply_rows(const int64_t* __restrict__ row, const int32_t* __restrict__ ptri,
                                                    const double* __restrict__ C, const double* __restrict__ f,
                                                    int64_t N, int d, int d0, int64_t M, double* __restrict__ u,
                                                    int nq_rt) {
    constexpr int U = 8;
    const int nq = NQ > 0 ? NQ : nq_rt;
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    double u0[D];
    if (lane < D) {
#pragma unroll
        for (int k = 0; k < D; k++)
            if (k == lane) u0[k] = d0 + k < d ? u[(int64_t)(d0 + k) * M + t] : 0.0;
    }
    // row-local 32-bit indexing: entry r of the row is node r % nq of pair r / nq
    const int64_t p0 = row[t];
    const int len = (int)((row[t + 1] - p0) * nq);
    const double* __restrict__ Crow = C + p0 * nq;
    const int32_t* __restrict__ prow = ptri + p0;
    double s[D];
#pragma unroll
    for (int k = 0; k < D; k++) s[k] = 0.0;
    for (int r = lane; r < len; r += 32 * U) {
        double c[U];
        int src[U];
#pragma unroll
        for (int i = 0; i < U; i++) {
            const int ri = r + 32 * i;
            const bool ok = ri < len;
            const int pl = ri / nq;
            c[i] = ok ? Crow[ri] : 0.0;
            src[i] = ok ? prow[pl] * nq + (ri - pl * nq) : 0;
        }
#pragma unroll
        for (int i = 0; i < U; i++)
#pragma unroll
            for (int k = 0; k < D; k++) s[k] = fma(c[i], f[(int64_t)(d0 + k) * N + src[i]], s[k]);
    }
#pragma unroll
    for (int k = 0; k < D; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    }
    if (lane < D) {
#pragma unroll
        for (int k = 0; k < D; k++)
            if (k == lane && d0 + k < d) u[(int64_t)(d0 + k) * M + t] = u0[k] + s[k];
    }
}

// Float-float apply (mixed precision): weights and densities as pairs of FP32
// values (h + l, ~2^-48 relative), products split exactly, sums kept as
// (two-sum hi, FP32 error) pairs; GB300's FP64 FMA rate (2 per SM per clock)
// would otherwise bound the apply at one DFMA per weight entry.
// Entries in flight per lane and resident blocks per SM of the float-float
// apply (timed on the 16,384-triangle star: 4 and 8 give 0.28 ms against
// 0.36 ms for 8 and 4).
#ifndef VP_APPLY_U
#define VP_APPLY_U 4
#endif
#ifndef VP_APPLY_MINB
#define VP_APPLY_MINB 8
#endif
template <int NQ, int D>
__global__ void __launch_bounds__(256, D <= 2 ? VP_APPLY_MINB : 2) k_apply_rows_f2(const int64_t* __restrict__ row, const int32_t* __restrict__ ptri,
                                                       const float2* __restrict__ C2, const float2* __restrict__ f2v,
                                                       int64_t N, int d, int d0, int64_t M, double* __restrict__ u) {
    constexpr int U = VP_APPLY_U;
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    double u0[D];
    if (lane < D) {
#pragma unroll
        for (int k = 0; k < D; k++)
            if (k == lane) u0[k] = d0 + k < d ? u[(int64_t)(d0 + k) * M + t] : 0.0;
    }
    const int64_t p0 = row[t];
    const int len = (int)((row[t + 1] - p0) * NQ);
    const float2* __restrict__ Crow = C2 + p0 * NQ;
    const int32_t* __restrict__ prow = ptri + p0;
    float ah[D], al[D];
#pragma unroll
    for (int k = 0; k < D; k++) ah[k] = al[k] = 0.f;
    for (int r = lane; r < len; r += 32 * U) {
        float2 c[U];
        int src[U];
#pragma unroll
        for (int i = 0; i < U; i++) {
            const int ri = r + 32 * i;
            const bool ok = ri < len;
            const int pl = ri / NQ;
            c[i] = ok ? Crow[ri] : make_float2(0.f, 0.f);
            src[i] = ok ? prow[pl] * NQ + (ri - pl * NQ) : 0;
        }
#pragma unroll
        for (int i = 0; i < U; i++)
#pragma unroll
            for (int k = 0; k < D; k++) {
                const float2 fv = f2v[(int64_t)(d0 + k) * N + src[i]];
                const float p = __fmul_rn(c[i].x, fv.x);
                float e = __fmaf_rn(c[i].x, fv.x, -p);
                e = __fmaf_rn(c[i].x, fv.y, __fmaf_rn(c[i].y, fv.x, e));
                const float sm = __fadd_rn(ah[k], p);
                const float bb = __fsub_rn(sm, ah[k]);
                const float er = __fadd_rn(__fsub_rn(ah[k], __fsub_rn(sm, bb)), __fsub_rn(p, bb));
                ah[k] = sm;
                al[k] = __fadd_rn(al[k], __fadd_rn(er, e));
            }
    }
#pragma unroll
    for (int k = 0; k < D; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, ah[k], o), ol = __shfl_xor_sync(0xffffffffu, al[k], o);
            const float sm = __fadd_rn(ah[k], oh);
            const float bb = __fsub_rn(sm, ah[k]);
            const float er = __fadd_rn(__fsub_rn(ah[k], __fsub_rn(sm, bb)), __fsub_rn(oh, bb));
            ah[k] = sm;
            al[k] = __fadd_rn(__fadd_rn(al[k], ol), er);
        }
    }
    if (lane < D) {
#pragma unroll
        for (int k = 0; k < D; k++)
            if (k == lane && d0 + k < d) u[(int64_t)(d0 + k) * M + t] = u0[k] + ((double)ah[k] + (double)al[k]);
    }
}

// out[i] = (h, l) with h = fl32(x[i]), l = fl32(x[i] - h)
__global__ void k_to_f2(const double* __restrict__ x, int64_t n, float2* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float h = __double2float_rn(v);
    out[i] = make_float2(h, __double2float_rn(v - (double)h));
}

// fT[j][k] = f[k][j] (node-major copy of the densities), 32 x 32 tiles.
__global__ void k_transpose_f(const double* __restrict__ f, int d, int64_t N, double* __restrict__ fT) {
    __shared__ double tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int k = k0 + r;
        const int64_t j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < d && j < N) ? f[(int64_t)k * N + j] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t j = j0 + r;
        const int k = k0 + threadIdx.x;
        if (j < N && k < d) fT[j * d + k] = tile[threadIdx.x][r];
    }
}

// Many densities: warp per target, densities across lanes (lane + 32 i); the
// warp loads 32 entries (weight, source node) at a time and broadcasts each,
// so every load of the node-major densities is one coalesced row.
template <int NQ, int DB>
__global__ void __launch_bounds__(256) k_apply_many(const int64_t* __restrict__ row, const int32_t* __restrict__ ptri,
                                                    const double* __restrict__ C, const double* __restrict__ fT,
                                                    int d, int64_t M, double* __restrict__ u, int nq_rt) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    const int nq = NQ > 0 ? NQ : nq_rt;
    const int64_t e0 = row[t] * nq, e1 = row[t + 1] * nq;
    double s[DB];
#pragma unroll
    for (int i = 0; i < DB; i++) s[i] = 0.0;
    for (int64_t base = e0; base < e1; base += 32) {
        const int n = (int)min((int64_t)32, e1 - base);
        double myc = 0.0;
        int64_t mysrc = 0;
        if (lane < n) {
            const int64_t e = base + lane;
            const int64_t p = e / nq;
            myc = C[e];
            mysrc = ((int64_t)ptri[p] * nq + (e - p * nq)) * d;
        }
        for (int j = 0; j < n; j++) {
            const double c = __shfl_sync(0xffffffffu, myc, j);
            const int64_t src = __shfl_sync(0xffffffffu, mysrc, j);
#pragma unroll
            for (int i = 0; i < DB; i++) {
                const int k = lane + 32 * i;
                if (k < d) s[i] += c * fT[src + k];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < DB; i++) {
        const int k = lane + 32 * i;
        if (k < d) u[(int64_t)k * M + t] += s[i];
    }
}

template <int NQ>
void apply_rows(const int64_t* row, const int32_t* ptri, const double* C, const double* f, int64_t N, int d,
                int64_t M, double* u, int nq, cudaStream_t s) {
    const unsigned grid = (unsigned)((M * 32 + 255) / 256);
    for (int d0 = 0; d0 < d;) {
        const int D = pick_chunk(d - d0);
        switch (D) {
            case 8: k_apply_rows<NQ, 8><<<grid, 256, 0, s>>>(row, ptri, C, f, N, d, d0, M, u, nq); break;
            case 4: k_apply_rows<NQ, 4><<<grid, 256, 0, s>>>(row, ptri, C, f, N, d, d0, M, u, nq); break;
            case 2: k_apply_rows<NQ, 2><<<grid, 256, 0, s>>>(row, ptri, C, f, N, d, d0, M, u, nq); break;
            default: k_apply_rows<NQ, 1><<<grid, 256, 0, s>>>(row, ptri, C, f, N, d, d0, M, u, nq); break;
        }
        d0 += D;
    }
}

template <int NQ>
void apply_rows_f2(const int64_t* row, const int32_t* ptri, const float2* C2, const float2* f2v, int64_t N, int d,
                   int64_t M, double* u, cudaStream_t s) {
    const unsigned grid = (unsigned)((M * 32 + 255) / 256);
    for (int d0 = 0; d0 < d;) {
        const int D = pick_chunk(d - d0);
        switch (D) {
            case 8: k_apply_rows_f2<NQ, 8><<<grid, 256, 0, s>>>(row, ptri, C2, f2v, N, d, d0, M, u); break;
            case 4: k_apply_rows_f2<NQ, 4><<<grid, 256, 0, s>>>(row, ptri, C2, f2v, N, d, d0, M, u); break;
            case 2: k_apply_rows_f2<NQ, 2><<<grid, 256, 0, s>>>(row, ptri, C2, f2v, N, d, d0, M, u); break;
            default: k_apply_rows_f2<NQ, 1><<<grid, 256, 0, s>>>(row, ptri, C2, f2v, N, d, d0, M, u); break;
        }
        d0 += D;
    }
}

template <int NQ>
void apply_many(const int64_t* row, const int32_t* ptri, const double* C, const double* fT, int d, int64_t M,
                double* u, int nq, cudaStream_t s) {
    const unsigned grid = (unsigned)((M * 32 + 255) / 256);
    const int db = (d + 31) / 32;
    if (db <= 1) k_apply_many<NQ, 1><<<grid, 256, 0, s>>>(row, ptri, C, fT, d, M, u, nq);
    else if (db <= 2) k_apply_many<NQ, 2><<<grid, 256, 0, s>>>(row, ptri, C, fT, d, M, u, nq);
    else if (db <= 4) k_apply_many<NQ, 4><<<grid, 256, 0, s>>>(row, ptri, C, fT, d, M, u, nq);
    else k_apply_many<NQ, 8><<<grid, 256, 0, s>>>(row, ptri, C, fT, d, M, u, nq);
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


constexpr int FF_TPT = 2;   // targets per thread in the single-evaluation kernel

template <int D>
__global__ void __launch_bounds__(FF_THREADS) k_far_ff(const float* __restrict__ shi, const float* __restrict__ slo,
                                                       const float* __restrict__ q, int64_t N,
                                                       const float* __restrict__ thi, const float* __restrict__ tlo,
                                                       const int32_t* __restrict__ tnode, int64_t M, int d, int d0,
                                                       double* __restrict__ partial, int splits) {
    __shared__ FFSmem<D> sm;
    ff_load_table(sm);
    const int split = blockIdx.y;
    const int64_t per = (N + splits - 1) / splits;
    const int64_t j0 = split * per, j1 = min(N, j0 + per);
    const int64_t tbase = (int64_t)blockIdx.x * (FF_THREADS * FF_TPT) + threadIdx.x;
    ff_far_block<D, FF_TPT>(sm, shi, slo, q, j0, j1, thi, tlo, tnode, M, tbase, d, d0, partial + (int64_t)split * d * M);
}

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
                   const int32_t* tnode, int64_t M, double* partial, float* qbuf, int splits, cudaStream_t s,
                   float2* f2out, int nq) {
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
                k_prep_q_ff<1><<<pb, 256, 0, s>>>(W, f, N, d, d0, qbuf, d == 1 ? f2out : nullptr, nq);
                k_far_ff<1><<<grid, FF_THREADS, 0, s>>>(src.hi, src.lo, qbuf, N, tgt.hi, tgt.lo, tnode, M, d, d0, partial, splits);
                break;
        }
        d0 += D;
    }
}

void launch_reduce_splits(const double* partial, int splits, int64_t count, double* out, cudaStream_t s) {
    if (count > 0) k_reduce_splits<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(partial, splits, count, out);
}

size_t apply_ws_bytes(int64_t N, int d) { return d >= APPLY_MANY_MIN_D ? (size_t)N * d * sizeof(double) : 0; }

void launch_apply_fp64(const int64_t* row, const int32_t* ptri, const double* C, int nq, const double* f, int64_t N,
                       int d, int64_t M, double* u, double* fT, cudaStream_t s) {
    if (M <= 0) return;
    if (d >= APPLY_MANY_MIN_D && fT) {
        dim3 tg((unsigned)((N + 31) / 32), (unsigned)((d + 31) / 32)), tb(32, 8);
        k_transpose_f<<<tg, tb, 0, s>>>(f, d, N, fT);
        if (nq == 19) apply_many<19>(row, ptri, C, fT, d, M, u, nq, s);
        else if (nq == 16) apply_many<16>(row, ptri, C, fT, d, M, u, nq, s);
        else apply_many<0>(row, ptri, C, fT, d, M, u, nq, s);
    } else {
        if (nq == 19) apply_rows<19>(row, ptri, C, f, N, d, M, u, nq, s);
        else if (nq == 16) apply_rows<16>(row, ptri, C, f, N, d, M, u, nq, s);
        else apply_rows<0>(row, ptri, C, f, N, d, M, u, nq, s);
    }
}

void launch_to_f2(const double* x, int64_t n, float2* out, cudaStream_t s) {
    if (n > 0) k_to_f2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, out);
}

void launch_apply_f2(const int64_t* row, const int32_t* ptri, const float2* C2, int nq, const double* f, int64_t N,
                     int d, int64_t M, double* u, float2* f2v, cudaStream_t s) {
    if (M <= 0) return;
    launch_to_f2(f, (int64_t)d * N, f2v, s);
    if (nq == 19) apply_rows_f2<19>(row, ptri, C2, f2v, N, d, M, u, s);
    else apply_rows_f2<16>(row, ptri, C2, f2v, N, d, M, u, s);
}

void launch_ff_split(const double* xy, int64_t n, double ox, double oy, double q, FFCoords out, cudaStream_t s) {
    if (n > 0) k_ff_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, n, ox, oy, q, out.hi, out.lo);
}

// Loads this unit's log table on the current device (vp_create), and the
// kernels of the one-sided evaluation (far sums, split reduction, row apply):
// under lazy loading a kernel is otherwise loaded, possibly with a device
// allocation, at its first launch, which vp_potential_eval_noalloc must not do.
cudaError_t eval_module_prepare() {
    cudaError_t e = ensure_logtab();
    if (e != cudaSuccess) return e;
    const void* kernels[] = {
        (const void*)k_far_fp64<1>, (const void*)k_far_fp64<2>, (const void*)k_far_fp64<4>, (const void*)k_far_fp64<8>,
        (const void*)k_prep_q_ff<1>, (const void*)k_prep_q_ff<2>, (const void*)k_prep_q_ff<4>, (const void*)k_prep_q_ff<8>,
        (const void*)k_far_ff<1>, (const void*)k_far_ff<2>, (const void*)k_far_ff<4>, (const void*)k_far_ff<8>,
        (const void*)k_reduce_splits,
        (const void*)k_apply_rows<19, 1>, (const void*)k_apply_rows<19, 2>, (const void*)k_apply_rows<19, 4>,
        (const void*)k_apply_rows<19, 8>, (const void*)k_apply_rows<16, 1>, (const void*)k_apply_rows<16, 2>,
        (const void*)k_apply_rows<16, 4>, (const void*)k_apply_rows<16, 8>, (const void*)k_apply_rows<0, 1>,
        (const void*)k_apply_rows<0, 2>, (const void*)k_apply_rows<0, 4>, (const void*)k_apply_rows<0, 8>};
    for (const void* k : kernels) {
        cudaFuncAttributes a;
        e = cudaFuncGetAttributes(&a, k);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
