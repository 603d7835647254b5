// Correction apply on the tensor cores (the last sum of the subtract-and-add
// evaluation, Section 3.6) for many densities at once:
//
//   u[n][t] += sum_{(t,T) in lists} sum_k C[t,T,k] f[n][T nq + k].
//
// The block-sparse C (1 x nq blocks) is re-laid per tile of 128 targets in
// Morton order as a dense block row over the union of the tile's triangles
// (24 columns per triangle: the nq = 19 nodes and 5 or 8 zeros), near pairs
// and self pairs in two separate runs of columns (self weights are some 30x
// larger than near ones, so each run gets its own row exponent).  C and f are
// split exactly into L balanced base-128 digits (exponent per target and run
// for C, per density for f):
//
//   C[t,e] = 2^(e_t - 7L + 1) sum_s a_s 128^(L-1-s),  |a_s| <= 64,
//   f[n,e] = 2^(tau_n - 7L + 1) sum_r b_r 128^(L-1-r), |b_r| <= 64,
//
// up to the rounding of C and f to 7L - 1 bits below their run/density
// maximum.  Digits are integers, exact in bf16; the products a_s b_r are at
// most 2^12 and every level sum Acc_l = sum_{s+r=l} sum_e a_s b_r stays below
// 2^24 for up to 2^12 / L columns, so the FP32 accumulation of the tensor
// cores is exact.  With the f digits stacked along N (n' = r dn + n, dn
// densities per pass), one MMA with A = a_s writes a_s b_r into TMEM columns
// dn (s + r) + n: the level sums land in their own column blocks without any
// shuffling.  After each run of at most 2^12 / L columns the 2L - 1 blocks
// are read back and combined in float-float,
//   sum_l 2^(-7 l) Acc_l,
// and scaled by 2^(e_t + tau_n - 12) into FP64 u.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "vp_internal.h"
#include "vp_async.cuh"

namespace {

constexpr int TC_M = 128;          // targets per tile (MMA M)
constexpr int TC_DN = 64;          // most densities per pass (32 with 5 digits)
constexpr int TC_KPT = 24;         // K columns per triangle
constexpr int TC_CH_TRI = 2;       // triangles per K chunk
constexpr int TC_CH_K = TC_KPT * TC_CH_TRI;   // 48
constexpr int TC_KSTEPS = TC_CH_K / 16;        // 3 MMAs of K = 16 per digit per chunk
#ifndef VP_TC_KPS
#define VP_TC_KPS 3
#endif
constexpr int TC_KPS = VP_TC_KPS;                 // k-steps per pipeline stage (1 or 3: a whole chunk)
static_assert(TC_KPS == 1 || TC_KPS == TC_KSTEPS, "a stage is one k-step or a whole chunk");
constexpr int TC_STAGES = TC_KPS == 1 ? 8 : 3;    // stages that fit 227 KB of shared memory
constexpr int TC_THREADS = 192;   // producer warp, MMA warp, four epilogue warps
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_PAIR_CAP = 16384;  // near pairs per tile the plan can hold

// one row group (8 targets) of a chunk: [k-step][digit][2 column halves][8 rows x 16 B]
__host__ __device__ constexpr uint32_t a_group_bytes(int L) { return (uint32_t)L * TC_KSTEPS * 256u; }
// one k-step of a row group: [digit][2 column halves][8 rows x 16 B]
__host__ __device__ constexpr uint32_t a_gstep_bytes(int L) { return (uint32_t)L * 256u; }
__host__ __device__ constexpr int dens_per_pass(int L) { return L <= 4 ? 64 : 32; }   // dn (2L - 1) <= 512 columns
__host__ __device__ constexpr uint32_t b_step_bytes(int L) { return (uint32_t)L * dens_per_pass(L) * 16u * 2u; }
// a pipeline stage: one k-step of a chunk, the 16 row groups of weight digits
// and the density digits of its 16 columns
__host__ __device__ constexpr uint32_t stage_bytes_of(int L) {
    return TC_KPS * (16u * a_gstep_bytes(L) + b_step_bytes(L));
}
// chunks per exact FP32 accumulation: K L 2^12 < 2^24
__host__ __device__ constexpr int super_chunks(int L) { return (1 << 24) / (L * 4096 * TC_CH_K); }

// ------------------------------------------------------------ plan: order
__device__ __forceinline__ uint32_t spread16(uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// key = Morton code of the target on a 2^16 grid over the box (clamped) << 32 | t
__global__ void k_morton_keys(const double* __restrict__ txy, int64_t M, int64_t n2, double x0, double y0,
                              double sx, double sy, unsigned long long* __restrict__ keys) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n2) return;
    if (t >= M) {
        keys[t] = ~0ULL;
        return;
    }
    const double gx = fmin(fmax((txy[2 * t] - x0) * sx, 0.0), 65535.0);
    const double gy = fmin(fmax((txy[2 * t + 1] - y0) * sy, 0.0), 65535.0);
    const uint32_t code = spread16((uint32_t)gx) | (spread16((uint32_t)gy) << 1);
    keys[t] = ((unsigned long long)code << 32) | (unsigned long long)t;
}

// Bitonic sort of n2 = 2^m keys: a global step for strides >= 1024, a
// shared-memory kernel for the rest of each merge.
__global__ void k_bitonic_global(unsigned long long* __restrict__ a, int64_t n2, int64_t k, int64_t j) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const int64_t l = i ^ j;
    if (l > i) {
        const unsigned long long x = a[i], y = a[l];
        const bool up = (i & k) == 0;
        if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
        }
    }
}

// merges of size <= k with strides j0, j0/2, ..., 1 inside blocks of 2048
__global__ void __launch_bounds__(1024) k_bitonic_shared(unsigned long long* __restrict__ a, int64_t n2, int64_t kmin,
                                                         int64_t kmax, int64_t jstart) {
    __shared__ unsigned long long s[2048];
    const int64_t base = (int64_t)blockIdx.x * 2048;
    for (int i = threadIdx.x; i < 2048; i += 1024) s[i] = base + i < n2 ? a[base + i] : ~0ULL;
    __syncthreads();
    for (int64_t k = kmin; k <= kmax; k <<= 1) {
        for (int64_t j = (k == kmin && jstart > 0) ? jstart : (k >> 1); j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < 2048; i += 1024) {
                const int l = i ^ (int)j;
                if (l > i) {
                    const unsigned long long x = s[i], y = s[l];
                    const bool up = ((base + i) & k) == 0;
                    if ((x > y) == up) {
                        s[i] = y;
                        s[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < 2048; i += 1024)
        if (base + i < n2) a[base + i] = s[i];
}

__global__ void k_perm_from_keys(const unsigned long long* __restrict__ keys, int64_t M, int64_t n_slots,
                                 int32_t* __restrict__ perm, int32_t* __restrict__ pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    if (i < M) {
        const int32_t t = (int32_t)(keys[i] & 0xffffffffULL);
        perm[i] = t;
        pos[t] = (int32_t)i;
    } else {
        perm[i] = -1;
    }
}

// ------------------------------------------------------------ plan: tiles
// Block per tile: the sorted unions of the triangles of its targets' near
// pairs and of its self pairs (keys tri and tri + 2^30).  Pass 0 writes the
// chunk counts (0 and an overflow flag when the pairs exceed the cap); pass 1
// writes the near union then the self union, two triangles per chunk (an odd
// tail repeats the last one, whose weights there are zero), and the slot of
// every pair (self slots after all near chunks).
constexpr int32_t SELF_KEY = 1 << 30;

__global__ void __launch_bounds__(512) k_tile_union(const int32_t* __restrict__ perm, const int64_t* __restrict__ row,
                                                    const int32_t* __restrict__ ptri, const uint8_t* __restrict__ pkind,
                                                    int pass, int32_t* __restrict__ ucount,
                                                    int32_t* __restrict__ ucount_near,
                                                    const int64_t* __restrict__ chunk_ptr,
                                                    int32_t* __restrict__ chunk_tri, int32_t* __restrict__ pslot,
                                                    int32_t* __restrict__ flag) {
    extern __shared__ int32_t su[];
    int32_t* keys = su;                        // [TC_PAIR_CAP]
    int32_t* uniq = su + TC_PAIR_CAP;          // [TC_PAIR_CAP]
    __shared__ int64_t off[TC_M + 1];
    __shared__ int64_t rbeg[TC_M];
    __shared__ int wsum[16];
    __shared__ int n_uniq, n_near_u;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (tid < TC_M) {
        const int32_t t = perm[(int64_t)b * TC_M + tid];
        rbeg[tid] = t >= 0 ? row[t] : 0;
        off[tid + 1] = t >= 0 ? row[t + 1] - row[t] : 0;
    }
    __syncthreads();
    if (tid == 0) {
        off[0] = 0;
        for (int i = 0; i < TC_M; i++) off[i + 1] += off[i];
    }
    __syncthreads();
    const int64_t total = off[TC_M];
    if (total > TC_PAIR_CAP) {
        if (tid == 0) {
            if (pass == 0) ucount[b] = ucount_near[b] = 0;
            atomicOr(flag, 1);
        }
        return;
    }
    int n2 = 2;
    while (n2 < total) n2 <<= 1;
    for (int j = tid; j < n2; j += blockDim.x) {
        int32_t key = INT32_MAX;
        if (j < total) {
            int lo = 0, hi = TC_M - 1;             // row i with off[i] <= j < off[i+1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= j) lo = mid;
                else hi = mid - 1;
            }
            const int64_t p = rbeg[lo] + (j - off[lo]);
            key = ptri[p] + (pkind[p] ? SELF_KEY : 0);
        }
        keys[j] = key;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t x = keys[i], y = keys[l];
                    if ((x > y) == ((i & k) == 0)) {
                        keys[i] = y;
                        keys[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    // compaction of the distinct keys: each thread a contiguous run
    const int per = (n2 + blockDim.x - 1) / blockDim.x;
    const int j0 = tid * per, j1 = min(n2, j0 + per);
    int cnt = 0, cnt_near = 0;
    for (int j = j0; j < j1; j++) {
        const bool first = keys[j] != INT32_MAX && (j == 0 || keys[j] != keys[j - 1]);
        cnt += first;
        cnt_near += first && keys[j] < SELF_KEY;
    }
    // block exclusive scan of cnt; total of cnt_near
    const int lane = tid & 31, w = tid >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int near_w = cnt_near;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) near_w += __shfl_xor_sync(0xffffffffu, near_w, o);
    if (tid == 0) n_near_u = 0;
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (lane == 0) atomicAdd(&n_near_u, near_w);
    if (tid == 0) {
        int acc = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            const int v = wsum[i];
            wsum[i] = acc;
            acc += v;
        }
        n_uniq = acc;
    }
    __syncthreads();
    int at = wsum[w] + incl - cnt;
    for (int j = j0; j < j1; j++)
        if (keys[j] != INT32_MAX && (j == 0 || keys[j] != keys[j - 1])) uniq[at++] = keys[j];
    __syncthreads();
    const int nu = n_uniq, nn = n_near_u, ns = nu - nn;
    const int cn = (nn + TC_CH_TRI - 1) / TC_CH_TRI, cs = (ns + TC_CH_TRI - 1) / TC_CH_TRI;
    if (pass == 0) {
        if (tid == 0) {
            ucount[b] = cn + cs;
            ucount_near[b] = cn;
        }
        return;
    }
    const int64_t cbase = chunk_ptr[b];
    for (int i = tid; i < cn * TC_CH_TRI; i += blockDim.x) chunk_tri[cbase * TC_CH_TRI + i] = uniq[min(i, nn - 1)];
    for (int i = tid; i < cs * TC_CH_TRI; i += blockDim.x)
        chunk_tri[(cbase + cn) * TC_CH_TRI + i] = uniq[nn + min(i, ns - 1)] - SELF_KEY;
    for (int64_t j = tid; j < total; j += blockDim.x) {
        int lo = 0, hi = TC_M - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= j) lo = mid;
            else hi = mid - 1;
        }
        const int64_t p = rbeg[lo] + (j - off[lo]);
        const int32_t key = ptri[p] + (pkind[p] ? SELF_KEY : 0);
        int a = 0, c = nu - 1;                     // position of key in uniq
        while (a < c) {
            const int mid = (a + c) >> 1;
            if (uniq[mid] < key) a = mid + 1;
            else c = mid;
        }
        pslot[p] = a < nn ? a : cn * TC_CH_TRI + (a - nn);
    }
}

// ------------------------------------------------------------ digits
// Balanced base-128 digits of X, |X| <= 2^(7L-1): X = sum_s a_s 128^(L-1-s),
// a_s in [-64, 63] for s >= 1 and a_0 in [-64, 64].
constexpr int TC_LMAX = 5;
__device__ __forceinline__ void digits128(long long X, int L, int (&a)[TC_LMAX]) {
#pragma unroll
    for (int s = TC_LMAX - 1; s >= 1; s--) {
        if (s < L) {
            const int r = (int)(((X + 64) & 127) - 64);
            a[s] = r;
            X = (X - r) >> 7;
        } else {
            a[s] = 0;
        }
    }
    a[0] = (int)X;
}

__device__ __forceinline__ uint16_t bf16_bits(int v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));   // |v| <= 64: exact
}

// exponent e with max < 2^e (0 for max = 0): frexp's
__device__ __forceinline__ int exp_above(double m) {
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    return e;
}

// warp per target: exponents of max |C| over its near entries and over its
// self entries (rexp[t], rexp[M + t])
template <int NQ>
__global__ void k_row_exp(const int64_t* __restrict__ row, const uint8_t* __restrict__ pkind,
                          const double* __restrict__ C, int64_t M, int32_t* __restrict__ rexp) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    double mn = 0.0, ms = 0.0;
    for (int64_t e = row[t] * NQ + lane; e < row[t + 1] * NQ; e += 32) {
        const double v = fabs(C[e]);
        if (pkind[e / NQ]) ms = fmax(ms, v);
        else mn = fmax(mn, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmax(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        ms = fmax(ms, __shfl_xor_sync(0xffffffffu, ms, o));
    }
    if (lane == 0) {
        rexp[t] = exp_above(mn);
        rexp[M + t] = exp_above(ms);
    }
}

// warp per target: digits of its weights scattered into the dense A images
// (per chunk: [digit s][k-step][16 row groups x 2 column halves][8 rows x 16 B])
// warp per target: the row group of the target in its tile, marked in every
// chunk that holds one of its pairs
__global__ void k_group_mask(const int64_t* __restrict__ row, const int32_t* __restrict__ pslot,
                             const int32_t* __restrict__ pos, const int64_t* __restrict__ chunk_ptr, int64_t M,
                             uint32_t* __restrict__ gmask) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    const int ps = pos[t];
    const int b = ps / TC_M, i = ps % TC_M;
    const int64_t cb = chunk_ptr[b];
    for (int64_t p = row[t] + lane; p < row[t + 1]; p += 32) atomicOr(&gmask[cb + pslot[p] / TC_CH_TRI], 1u << (i >> 3));
}

__global__ void k_popc(const uint32_t* __restrict__ m, int64_t n, int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = __popc(m[i]);
}

template <int NQ>
__global__ void k_scatter_a(const int64_t* __restrict__ row, const uint8_t* __restrict__ pkind,
                            const double* __restrict__ C, const int32_t* __restrict__ pslot,
                            const int32_t* __restrict__ pos, const int64_t* __restrict__ chunk_ptr,
                            const uint32_t* __restrict__ gmask, const int64_t* __restrict__ gptr,
                            const int32_t* __restrict__ rexp, int64_t M, int L, uint16_t* __restrict__ A) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= M) return;
    const int ps = pos[t];
    const int b = ps / TC_M, i = ps % TC_M;
    const int64_t cb = chunk_ptr[b];
    if (chunk_ptr[b + 1] == cb) return;             // no pairs
    const int sh_near = 7 * L - 1 - rexp[t], sh_self = 7 * L - 1 - rexp[M + t];
    const size_t gbytes = a_group_bytes(L);
    const int g = i >> 3;
    const int64_t e0 = row[t] * NQ, e1 = row[t + 1] * NQ;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int64_t p = e / NQ;
        const int k = (int)(e - p * NQ);
        const int slot = pslot[p];
        const int64_t chunk = cb + slot / TC_CH_TRI;
        const int kk = (slot % TC_CH_TRI) * TC_KPT + k;
        const int ks = kk >> 4, kc = kk & 15;
        const long long X = __double2ll_rn(ldexp(C[e], pkind[p] ? sh_self : sh_near));
        int a[TC_LMAX];
        digits128(X, L, a);
        const int64_t blk = gptr[chunk] + __popc(gmask[chunk] & ((1u << g) - 1u));   // stored row group
        const size_t base = (size_t)blk * gbytes + (size_t)(kc >> 3) * 128 + (size_t)(i & 7) * 16 + (size_t)(kc & 7) * 2;
#pragma unroll
        for (int s = 0; s < TC_LMAX; s++)
            if (s < L) A[(base + (size_t)(ks * L + s) * 256) / 2] = bf16_bits(a[s]);
    }
}

// |f| maxima per density of the pass (as the bits of a non-negative double)
__global__ void k_fmax(const double* __restrict__ f, int64_t N, int d, int d0, unsigned long long* __restrict__ fmaxb) {
    const int n = blockIdx.y;
    if (d0 + n >= d) return;
    double m = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(f[(int64_t)(d0 + n) * N + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&fmaxb[n], (unsigned long long)__double_as_longlong(m));
}

// density digits: B[(r dn + n) nT + T][24] bf16 (nodes past nq zero)
template <int NQ>
__global__ void k_fdigits(const double* __restrict__ f, int64_t N, int64_t nT, int d, int d0, int L, int dn,
                          const unsigned long long* __restrict__ fmaxb, uint16_t* __restrict__ B) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nT * dn) return;
    const int n = (int)(gid / nT);
    const int64_t T = gid - (int64_t)n * nT;
    const bool live = d0 + n < d;
    const int tau = live ? exp_above(__longlong_as_double((long long)fmaxb[n])) : 0;
    const int sh = 7 * L - 1 - tau;
    uint32_t w[TC_LMAX][TC_KPT / 2];
#pragma unroll
    for (int k2 = 0; k2 < TC_KPT / 2; k2++) {
        int lo[TC_LMAX] = {0, 0, 0, 0, 0}, hi[TC_LMAX] = {0, 0, 0, 0, 0};
        const int ka = 2 * k2, kb = 2 * k2 + 1;
        if (live && ka < NQ) digits128(__double2ll_rn(ldexp(f[(int64_t)(d0 + n) * N + T * NQ + ka], sh)), L, lo);
        if (live && kb < NQ) digits128(__double2ll_rn(ldexp(f[(int64_t)(d0 + n) * N + T * NQ + kb], sh)), L, hi);
#pragma unroll
        for (int r = 0; r < TC_LMAX; r++) w[r][k2] = (uint32_t)bf16_bits(lo[r]) | ((uint32_t)bf16_bits(hi[r]) << 16);
    }
#pragma unroll
    for (int r = 0; r < TC_LMAX; r++) {
        if (r >= L) break;
        uint4* dst = (uint4*)(B + ((size_t)(r * dn + n) * nT + T) * TC_KPT);
#pragma unroll
        for (int v = 0; v < 3; v++) dst[v] = make_uint4(w[r][4 * v], w[r][4 * v + 1], w[r][4 * v + 2], w[r][4 * v + 3]);
    }
}

// ------------------------------------------------------------ tcgen05 glue
// zeros for the row groups a stage must clear (copied like data, so that no
// generic-proxy store has to be fenced before the tensor cores read the stage)
__device__ __align__(128) unsigned char g_tc_zero[4096];

// tiled TMA load of a 3-D box at (x, y, z) into shared memory, completing on an mbarrier
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor, no swizzle, K-major core matrices of
// 8 rows x 16 B: lbo = byte step between the two K halves of a 16-wide
// k-step, sbo = byte step between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ULL << 46);
}
// instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16_zero(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct TcArgs {
    const int32_t* perm;        // [n_tiles * 128]
    const int64_t* chunk_ptr;   // [n_tiles + 1]
    const int32_t* chunk_near;  // [n_tiles] near chunks of each tile (self chunks follow)
    const int32_t* chunk_tri;   // [n_chunks][2]
    const int32_t* rexp;        // [2][M] near and self row exponents
    const uint16_t* A;          // [stored row groups] digit images
    const uint32_t* gmask;      // [n_chunks] stored row groups of each chunk
    const int64_t* gptr;        // [n_chunks] first stored row group of each chunk
    const uint16_t* B;          // [L dn][nT][24] density digits
    const unsigned long long* fmaxb;   // [dn]
    int64_t nT, M, n_tiles;
    int L, dn, d, d0;
    int32_t* flag;              // device error flags
    double* u;                  // [d][M]
};

__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Chunk c of a tile with n_near near chunks and nch in all: its run (near or
// self, cut every sc chunks) and whether it opens or closes that run.
struct ChunkPos {
    bool self_run, first, last;
};
__device__ __forceinline__ ChunkPos chunk_pos(int64_t c, int64_t n_near, int64_t nch, int sc) {
    ChunkPos r;
    r.self_run = c >= n_near;
    const int64_t pos = r.self_run ? c - n_near : c, len = r.self_run ? nch - n_near : n_near;
    r.first = (pos % sc) == 0;
    r.last = (pos % sc) == sc - 1 || pos == len - 1;
    return r;
}

// Persistent and warp-specialised: one CTA per SM walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... (Morton order, so neighbouring
// tiles have similar chunk counts).
//   warp 0 (producer): per chunk, waits for the stage to be free, zeroes the
//     row groups the stage still holds from an earlier chunk, and issues the
//     copies: the chunk's stored row groups of weight digits (bulk copies)
//     and its two triangles' density digits (six TMA tensor boxes), all
//     completing on the stage's full barrier;
//   warp 1 (MMA): per chunk, waits for the stage, issues the L x 3 MMAs and
//     commits them to the stage's empty barrier; at the end of a run it
//     commits to acc_full and, before the next run, waits for acc_empty;
//   warps 2-5 (epilogue, TMEM lanes 32 (w mod 4) ..): zero the accumulator
//     columns, and after each run read the level sums, combine them in
//     float-float and add them to u, zero the columns again and arrive on
//     acc_empty.
// No CTA-wide barrier inside the loop; every wait is bounded and an abort
// (a wait that gave up) is shared through shared memory, drained, reported.
template <int DN>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_apply(TcArgs a, const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    const int L = a.L;
    constexpr int dn = DN;   // densities per pass (dens_per_pass(L))
    // stage: [16 row groups][TC_KPS k-steps][L digits][2 halves][8 rows x 16 B], then
    // [TC_KPS k-steps][2 halves][L dn density rows x 16 B]
    const uint32_t gstep = a_gstep_bytes(L), gst = TC_KPS * gstep, abytes = 16u * gst, bstep = b_step_bytes(L);
    const uint32_t stage_bytes = stage_bytes_of(L);
    uint64_t* bars = (uint64_t*)(base + TC_STAGES * stage_bytes);   // full[S], empty[S], acc_full, acc_empty
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * TC_STAGES + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    int* tau = (int*)(tmem_slot + 2);                                // [dn]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(base);
    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[TC_STAGES + s]); };
    const uint32_t acc_full = smem_u32(&bars[2 * TC_STAGES]), acc_empty = smem_u32(&bars[2 * TC_STAGES + 1]);

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; s++) {
            mbar_init(full_bar(s), 1);     // lane 0's expect_tx arrival; the copies complete the transactions
            mbar_init(empty_bar(s), 1);    // the MMA warp's commit
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 4);           // one arrival per epilogue warp
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (tid < dn) tau[tid] = a.d0 + tid < a.d ? exp_above(__longlong_as_double((long long)a.fmaxb[tid])) : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nlev = 2 * L - 1;
    const int sc = super_chunks(L);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // Per k-step of a chunk (one stage): the k-step of its stored row
        // groups of weight digits (bulk copies, lanes 0-15) and the density
        // digits of its two column halves (TMA boxes of L dn rows x 16 B, lanes
        // 16-17), all completing on the stage's full barrier; row groups the
        // stage still holds from an earlier chunk are zeroed first.  Chunk
        // metadata is loaded 32 chunks at a time.
        const uint32_t gbytes = a_group_bytes(L);
        const uint32_t kbox = (uint32_t)(L * dn) * 16u;   // one density-digit box
        uint32_t held[TC_STAGES];          // row groups each stage holds nonzero digits of (unknown at first)
#pragma unroll
        for (int s = 0; s < TC_STAGES; s++) held[s] = 0xFFFFu;
        uint32_t k = 0;                    // stages issued
        bool ok = true;
        for (int64_t b = blockIdx.x; b < a.n_tiles && ok; b += gridDim.x) {
            const int64_t c0 = a.chunk_ptr[b], nch = a.chunk_ptr[b + 1] - c0;
            int32_t mt0 = 0, mt1 = 0;
            uint32_t mm = 0;
            int64_t mg = 0;
            for (int64_t c = 0; c < nch; c++) {
                if ((c & 31) == 0) {       // metadata of the next 32 chunks, one per lane
                    const int64_t cc = c0 + c + lane;
                    if (c + lane < nch) {
                        mt0 = a.chunk_tri[2 * cc];
                        mt1 = a.chunk_tri[2 * cc + 1];
                        mm = a.gmask[cc];
                        mg = a.gptr[cc];
                    }
                }
                const int src = (int)(c & 31);
                const int32_t t0 = __shfl_sync(0xffffffffu, mt0, src), t1 = __shfl_sync(0xffffffffu, mt1, src);
                const uint32_t m = __shfl_sync(0xffffffffu, mm, src);
                const int64_t gp = __shfl_sync(0xffffffffu, mg, src);
                for (int ks = 0; ks < TC_KSTEPS && ok; ks += TC_KPS) {
                    const int s = (int)(k % TC_STAGES);
                    int stop = 0;                  // decided by lane 0, the same for the whole warp
                    if (lane == 0) {
                        stop = *abort_flag;
                        if (!stop && k >= TC_STAGES && !mbar_wait(empty_bar(s), ((k / TC_STAGES) - 1) & 1)) {
                            stop = 1;
                            *abort_flag = 1;
                        }
                    }
                    if (__shfl_sync(0xffffffffu, stop, 0)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = sbase + s * stage_bytes, sb = sa + abytes;
                    uint32_t z = 0;
#pragma unroll
                    for (int q = 0; q < TC_STAGES; q++)
                        if (q == s) {
                            z = held[q] & ~m;
                            held[q] = m;
                        }
                    if (lane == 0) mbar_expect_tx(full_bar(s), (uint32_t)__popc(m | z) * gst + 2u * TC_KPS * kbox);
                    __syncwarp();
                    if (lane < 16) {
                        if ((m >> lane) & 1u)
                            bulk_g2s(sa + lane * gst,
                                     (const unsigned char*)a.A +
                                         (size_t)(gp + __popc(m & ((1u << lane) - 1u))) * gbytes + ks * gstep,
                                     gst, full_bar(s));
                        else if ((z >> lane) & 1u)
                            bulk_g2s(sa + lane * gst, g_tc_zero, gst, full_bar(s));
                    } else if (lane < 16 + 2 * TC_KPS) {
                        // column half h of k-step ks + j: column group kg = 2 (ks + j) + h,
                        // triangle kg / 3, columns 8 (kg % 3) .. + 7
                        const int j = (lane - 16) >> 1, h = (lane - 16) & 1, kg = 2 * (ks + j) + h;
                        tma_load3(sb + j * bstep + h * (bstep / 2), &tmB, 8 * (kg % 3), kg < 3 ? t0 : t1, 0,
                                  full_bar(s));
                    }
                    k++;
                }
                if (!ok) break;
            }
        }
        // after an abort: the copies still in flight into the stages
        if (!ok && lane == 0)
            for (uint32_t j = k > TC_STAGES ? k - TC_STAGES : 0; j < k; j++)
                mbar_wait(full_bar((int)(j % TC_STAGES)), (j / TC_STAGES) & 1);
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_M, dn * L);
            uint32_t k = 0, runs = 0;
            bool ok = true;
            for (int64_t b = blockIdx.x; b < a.n_tiles && ok; b += gridDim.x) {
                const int64_t c0 = a.chunk_ptr[b], nch = a.chunk_ptr[b + 1] - c0, n_near = a.chunk_near[b];
                for (int64_t c = 0; c < nch; c++) {
                    const ChunkPos cp = chunk_pos(c, n_near, nch, sc);
                    if (*abort_flag || (cp.first && !mbar_wait(acc_empty, runs & 1))) {
                        ok = false;
                        *abort_flag = 1;
                        break;
                    }
                    for (int ks = 0; ks < TC_KSTEPS; ks += TC_KPS) {
                        const int s = (int)(k % TC_STAGES);
                        if (!mbar_wait(full_bar(s), (k / TC_STAGES) & 1)) {
                            ok = false;
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = sbase + s * stage_bytes, sb = sa + abytes;
#pragma unroll
                        for (int j = 0; j < TC_KPS; j++) {
                            // density rows 16 B apart (8-row groups 128 B apart), the column halves bstep / 2 apart
                            const uint64_t bdesc = smem_desc(sb + j * bstep, bstep / 2, 128);
                            for (int sd = 0; sd < L; sd++) {
                                // row groups gst apart, the two column halves 128 B apart
                                const uint64_t adesc = smem_desc(sa + j * gstep + sd * 256, 128, gst);
                                mma_bf16(tmem + dn * sd, adesc, bdesc, idesc, 1u);
                            }
                        }
                        mma_commit(empty_bar(s));
                        k++;
                    }
                    if (!ok) break;
                    if (cp.last) {
                        mma_commit(acc_full);
                        runs++;
                    }
                }
            }
            if (k > 0) mbar_wait(empty_bar((int)((k - 1) % TC_STAGES)), ((k - 1) / TC_STAGES) & 1);
            if (!ok) atomicOr(a.flag, VP_DEV_ERR_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;                                      // TMEM lane quarter of this warp
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int row = q * 32 + lane;
        auto zero_acc = [&]() {
            for (int l = 0; l < nlev; l++)
                for (int g = 0; g < dn / 16; g++) tmem_st16_zero(tmem + lane_base + dn * l + 16 * g);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(acc_empty);
        };
        zero_acc();
        uint32_t runs = 0;
        bool ok = true;
        for (int64_t b = blockIdx.x; b < a.n_tiles && ok; b += gridDim.x) {
            const int64_t c0 = a.chunk_ptr[b], nch = a.chunk_ptr[b + 1] - c0, n_near = a.chunk_near[b];
            const int32_t t = a.perm[b * TC_M + row];
            // with 32 densities per pass this tile's corrections of the target
            // are summed over its runs in registers (FP64) and written once
            constexpr int NACC = DN == 32 ? 32 : 1;
            double acc[NACC];
#pragma unroll
            for (int n = 0; n < NACC; n++) acc[n] = 0.0;
            double* ut = a.u + (int64_t)a.d0 * a.M + (t >= 0 ? t : 0);
            for (int64_t c = 0; c < nch; c++) {
                const ChunkPos cp = chunk_pos(c, n_near, nch, sc);
                if (!cp.last) continue;
                int stop = 0;
                if (lane == 0) stop = *abort_flag || !mbar_wait(acc_full, runs & 1);
                if (__shfl_sync(0xffffffffu, stop, 0)) {
                    ok = false;
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                // the level sums of this run, combined in float-float as they are read
                float H[DN], Lo[DN];
#pragma unroll
                for (int j = 0; j < DN; j++) H[j] = Lo[j] = 0.f;
                for (int l = 0; l < nlev; l++) {
                    const float scl = __int_as_float((127 - 7 * l) << 23);   // 2^(-7 l), exact
#pragma unroll
                    for (int g = 0; g < DN / 16; g++) {
                        uint32_t v[16];
                        tmem_ld16(tmem + lane_base + dn * l + 16 * g, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            float sm, er;
                            two_sum_f(H[16 * g + j], __fmul_rn(__int_as_float((int)v[j]), scl), sm, er);
                            H[16 * g + j] = sm;
                            Lo[16 * g + j] = __fadd_rn(Lo[16 * g + j], er);
                        }
                    }
                }
                // free the accumulator at once: the MMAs of the next run overlap the rest
                zero_acc();
                runs++;
                const int et = t >= 0 ? a.rexp[(cp.self_run ? a.M : 0) + t] - 12 : 0;
                if (DN == 32) {
#pragma unroll
                    for (int j = 0; j < NACC; j++) acc[j] += ldexp((double)H[j] + (double)Lo[j], et + tau[j]);
                } else if (t >= 0) {
                    // read-modify-write in groups of 8 densities: the loads first, then the stores
#pragma unroll
                    for (int j0 = 0; j0 < DN; j0 += 8) {
                        double old[8];
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            if (a.d0 + j0 + j < a.d) old[j] = ut[(int64_t)(j0 + j) * a.M];
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            if (a.d0 + j0 + j < a.d)
                                ut[(int64_t)(j0 + j) * a.M] =
                                    old[j] + ldexp((double)H[j0 + j] + (double)Lo[j0 + j], et + tau[j0 + j]);
                    }
                }
            }
            if constexpr (DN == 32) {
                if (!ok || t < 0) continue;
                // one read-modify-write per (target, density) and tile, in groups of 8 (loads, then stores)
#pragma unroll
                for (int j0 = 0; j0 < NACC; j0 += 8) {
                    double old[8];
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (a.d0 + j0 + j < a.d) old[j] = ut[(int64_t)(j0 + j) * a.M];
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (a.d0 + j0 + j < a.d) ut[(int64_t)(j0 + j) * a.M] = old[j] + acc[j0 + j];
                }
            }
        }
        if (!ok && lane == 0) atomicOr(a.flag, VP_DEV_ERR_TIMEOUT);
    }
    // all roles done (the MMA warp waited for its last commit): free TMEM
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

size_t tc_smem_bytes(int L) {
    return (size_t)TC_STAGES * stage_bytes_of(L) + 1024 + (2 * TC_STAGES + 2) * 8 + 8 + 4 * TC_DN;
}

}  // namespace

// ----------------------------------------------------------------- host
void tc_plan_free(TcPlan* p) {
    if (!p) return;
    cudaFree(p->d_perm);
    cudaFree(p->d_pos);
    cudaFree(p->d_chunk_ptr);
    cudaFree(p->d_chunk_tri);
    cudaFree(p->d_chunk_near);
    cudaFree(p->d_rexp);
    cudaFree(p->d_A);
    cudaFree(p->d_gmask);
    cudaFree(p->d_gptr);
    delete p;
}

int tc_plan_build(vp_ctx* ctx, vp_nf* nf, int L, cudaStream_t s) {
    if (L < 3 || L > TC_LMAX) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_nf_prepare_tc: levels must be 3, 4 or 5");
    const vp_mesh* mesh = nf->mesh;
    if (mesh->rule.builtin < 0)
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_nf_prepare_tc: the tensor-core apply takes the 16- and 19-node rules");
    const int64_t M = nf->M;
    const int nq = mesh->nq;
    TcPlan* p = new TcPlan();
    p->levels = L;
    p->n_tiles = (M + TC_M - 1) / TC_M;
    const int64_t n_slots = p->n_tiles * TC_M;
    int64_t n2 = 2048;
    while (n2 < M) n2 <<= 1;
    unsigned long long* keys = nullptr;
    int32_t* ucount = nullptr;
    int32_t* dflag = nullptr;
    int32_t* pslot = nullptr;
    int32_t* gcount = nullptr;
    auto fail = [&](int code, const char* msg) {
        cudaFree(keys);
        cudaFree(ucount);
        cudaFree(dflag);
        cudaFree(pslot);
        cudaFree(gcount);
        tc_plan_free(p);
        return vp_set_error(ctx, code, msg);
    };
#define TC_TRY(expr)                                                           \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess)                                                 \
            return fail(_e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA, \
                        "vp_nf_prepare_tc: " #expr);                           \
    } while (0)
    TC_TRY(cudaMalloc(&keys, n2 * sizeof(unsigned long long)));
    TC_TRY(cudaMalloc(&p->d_perm, n_slots * sizeof(int32_t)));
    TC_TRY(cudaMalloc(&p->d_pos, std::max<int64_t>(M, 1) * sizeof(int32_t)));
    TC_TRY(cudaMalloc(&ucount, (p->n_tiles + 1) * sizeof(int32_t)));
    TC_TRY(cudaMalloc(&p->d_chunk_near, (p->n_tiles + 1) * sizeof(int32_t)));
    TC_TRY(cudaMalloc(&p->d_chunk_ptr, (p->n_tiles + 1) * sizeof(int64_t)));
    TC_TRY(cudaMalloc(&dflag, sizeof(int32_t)));
    TC_TRY(cudaMalloc(&pslot, std::max<int64_t>(nf->P, 1) * sizeof(int32_t)));
    TC_TRY(cudaMalloc(&p->d_rexp, std::max<int64_t>(2 * M, 1) * sizeof(int32_t)));
    TC_TRY(cudaMemsetAsync(dflag, 0, sizeof(int32_t), s));
    // Morton order of the targets
    const double* bb = mesh->bbox;
    const double wx = std::max(bb[2] - bb[0], 1e-300), wy = std::max(bb[3] - bb[1], 1e-300);
    const double span = std::max(wx, wy) * 1.0000001;
    k_morton_keys<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(nf->d_txy, M, n2, bb[0], bb[1], 65536.0 / span,
                                                               65536.0 / span, keys);
    const unsigned sb = (unsigned)(n2 / 2048);
    k_bitonic_shared<<<sb, 1024, 0, s>>>(keys, n2, 2, 2048, 0);
    for (int64_t k = 4096; k <= n2; k <<= 1) {
        for (int64_t j = k >> 1; j >= 2048; j >>= 1)
            k_bitonic_global<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(keys, n2, k, j);
        k_bitonic_shared<<<sb, 1024, 0, s>>>(keys, n2, k, k, 1024);
    }
    k_perm_from_keys<<<(unsigned)((n_slots + 255) / 256), 256, 0, s>>>(keys, M, n_slots, p->d_perm, p->d_pos);
    TC_TRY(cudaGetLastError());
    // tiles: unions of triangles, chunk offsets, slots
    const size_t ush = 2 * TC_PAIR_CAP * sizeof(int32_t);
    TC_TRY(cudaFuncSetAttribute(k_tile_union, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ush));
    if (p->n_tiles > 0)
        k_tile_union<<<(unsigned)p->n_tiles, 512, ush, s>>>(p->d_perm, nf->d_row, nf->d_ptri, nf->d_pkind, 0, ucount,
                                                            p->d_chunk_near, nullptr, nullptr, nullptr, dflag);
    TC_TRY(cudaGetLastError());
    int32_t hflag = 0;
    TC_TRY(cudaMemcpyAsync(&hflag, dflag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaStreamSynchronize(s));
    if (hflag) return fail(VP_ERR_INVALID_ARG, "vp_nf_prepare_tc: a tile of 128 targets has more than 16384 near pairs");
    int rc = vp_exclusive_scan_i32(ctx, ucount, p->d_chunk_ptr, p->n_tiles, s);
    if (rc) return fail(rc, "vp_nf_prepare_tc: scan");
    TC_TRY(cudaMemcpyAsync(&p->n_chunks, p->d_chunk_ptr + p->n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaStreamSynchronize(s));
    TC_TRY(cudaMalloc(&p->d_chunk_tri, std::max<int64_t>(p->n_chunks, 1) * TC_CH_TRI * sizeof(int32_t)));
    if (p->n_tiles > 0)
        k_tile_union<<<(unsigned)p->n_tiles, 512, ush, s>>>(p->d_perm, nf->d_row, nf->d_ptri, nf->d_pkind, 1, ucount,
                                                            p->d_chunk_near, p->d_chunk_ptr, p->d_chunk_tri, pslot,
                                                            dflag);
    TC_TRY(cudaGetLastError());
    // which row groups (8 targets) of each chunk hold weights: only those are stored
    const unsigned wg = (unsigned)((M * 32 + 255) / 256);
    const int64_t nc1 = std::max<int64_t>(p->n_chunks, 1);
    TC_TRY(cudaMalloc(&p->d_gmask, nc1 * sizeof(uint32_t)));
    TC_TRY(cudaMalloc(&p->d_gptr, (nc1 + 1) * sizeof(int64_t)));
    TC_TRY(cudaMalloc(&gcount, nc1 * sizeof(int32_t)));
    TC_TRY(cudaMemsetAsync(p->d_gmask, 0, nc1 * sizeof(uint32_t), s));
    if (M > 0) k_group_mask<<<wg, 256, 0, s>>>(nf->d_row, pslot, p->d_pos, p->d_chunk_ptr, M, p->d_gmask);
    if (p->n_chunks > 0) k_popc<<<(unsigned)((p->n_chunks + 255) / 256), 256, 0, s>>>(p->d_gmask, p->n_chunks, gcount);
    TC_TRY(cudaGetLastError());
    rc = vp_exclusive_scan_i32(ctx, gcount, p->d_gptr, p->n_chunks, s);
    if (rc) return fail(rc, "vp_nf_prepare_tc: scan");
    TC_TRY(cudaMemcpyAsync(&p->n_groups, p->d_gptr + p->n_chunks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaStreamSynchronize(s));
    // weight digits of the stored row groups
    p->a_bytes = (size_t)p->n_groups * a_group_bytes(L);
    TC_TRY(cudaMalloc(&p->d_A, std::max<size_t>(p->a_bytes, 16)));
    TC_TRY(cudaMemsetAsync(p->d_A, 0, p->a_bytes, s));
    if (M > 0) {
        if (nq == 19) {
            k_row_exp<19><<<wg, 256, 0, s>>>(nf->d_row, nf->d_pkind, nf->d_C, M, p->d_rexp);
            k_scatter_a<19><<<wg, 256, 0, s>>>(nf->d_row, nf->d_pkind, nf->d_C, pslot, p->d_pos, p->d_chunk_ptr,
                                               p->d_gmask, p->d_gptr, p->d_rexp, M, L, p->d_A);
        } else {
            k_row_exp<16><<<wg, 256, 0, s>>>(nf->d_row, nf->d_pkind, nf->d_C, M, p->d_rexp);
            k_scatter_a<16><<<wg, 256, 0, s>>>(nf->d_row, nf->d_pkind, nf->d_C, pslot, p->d_pos, p->d_chunk_ptr,
                                               p->d_gmask, p->d_gptr, p->d_rexp, M, L, p->d_A);
        }
    }
    TC_TRY(cudaGetLastError());
    TC_TRY(cudaStreamSynchronize(s));
    cudaFree(keys);
    cudaFree(ucount);
    cudaFree(dflag);
    cudaFree(pslot);
    cudaFree(gcount);
#undef TC_TRY
    p->bytes = p->a_bytes + n_slots * 4 + M * 4 + (p->n_tiles + 1) * 12 + p->n_chunks * 20 + M * 8;
    tc_plan_free(nf->tc);
    nf->tc = p;
    return VP_OK;
}

size_t tc_ws_bytes(const vp_nf* nf) {
    if (!nf->tc) return 0;
    const int L = nf->tc->levels;
    const size_t bbytes = (size_t)L * dens_per_pass(L) * nf->mesh->nt * TC_KPT * sizeof(uint16_t);
    return ((bbytes + 255) & ~(size_t)255) + TC_DN * sizeof(unsigned long long) + 256;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

int tc_apply(vp_ctx* ctx, const vp_nf* nf, const double* f, int d, double* u, void* ws, cudaStream_t s) {
    const TcPlan* p = nf->tc;
    const vp_mesh* mesh = nf->mesh;
    const int L = p->levels, dn = dens_per_pass(L);
    const int64_t N = mesh->N, nT = mesh->nt;
    if (nf->M == 0 || p->n_chunks == 0) return VP_OK;
    const size_t bbytes = (size_t)L * dn * nT * TC_KPT * sizeof(uint16_t);
    uint16_t* B = (uint16_t*)ws;
    unsigned char* tail = (unsigned char*)ws + ((bbytes + 255) & ~(size_t)255);
    unsigned long long* fmaxb = (unsigned long long*)tail;                  // [dn]
    const size_t smem = tc_smem_bytes(L);
    // the density digits B[(r dn + n)][T][24] as a 3-D tensor (k, T, r dn + n) of
    // bf16; a box is 8 columns of one triangle for all L dn rows (16 B each)
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return vp_set_error(ctx, VP_ERR_CUDA, "tensor-core apply: cuTensorMapEncodeTiled unavailable");
    CUtensorMap tmB;
    const cuuint64_t gdim[3] = {(cuuint64_t)TC_KPT, (cuuint64_t)nT, (cuuint64_t)(L * dn)};
    const cuuint64_t gstride[2] = {(cuuint64_t)TC_KPT * 2, (cuuint64_t)nT * TC_KPT * 2};
    const cuuint32_t box[3] = {8, 1, (cuuint32_t)(L * dn)};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)B, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return vp_set_error(ctx, VP_ERR_CUDA, "tensor-core apply: cuTensorMapEncodeTiled failed");
    VP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_apply<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_apply<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>(p->n_tiles, ctx->sm_count);
    for (int d0 = 0; d0 < d; d0 += dn) {
        VP_CUDA_TRY(ctx, cudaMemsetAsync(tail, 0, TC_DN * sizeof(unsigned long long) + sizeof(int), s));
        dim3 mg(64, (unsigned)dn);
        k_fmax<<<mg, 256, 0, s>>>(f, N, d, d0, fmaxb);
        const unsigned fg = (unsigned)((nT * dn + 127) / 128);
        if (mesh->nq == 19) k_fdigits<19><<<fg, 128, 0, s>>>(f, N, nT, d, d0, L, dn, fmaxb, B);
        else k_fdigits<16><<<fg, 128, 0, s>>>(f, N, nT, d, d0, L, dn, fmaxb, B);
        TcArgs a;
        a.perm = p->d_perm;
        a.chunk_ptr = p->d_chunk_ptr;
        a.chunk_near = p->d_chunk_near;
        a.chunk_tri = p->d_chunk_tri;
        a.rexp = p->d_rexp;
        a.A = p->d_A;
        a.gmask = p->d_gmask;
        a.gptr = p->d_gptr;
        a.B = B;
        a.fmaxb = fmaxb;
        a.nT = nT;
        a.M = nf->M;
        a.n_tiles = p->n_tiles;
        a.L = L;
        a.dn = dn;
        a.d = d;
        a.d0 = d0;
        a.flag = ctx->d_flag;
        a.u = u;
        if (dn == 32) k_tc_apply<32><<<grid, TC_THREADS, smem, s>>>(a, tmB);
        else k_tc_apply<64><<<grid, TC_THREADS, smem, s>>>(a, tmB);
        VP_LAUNCH_CHECK(ctx);
    }
    return VP_OK;
}
