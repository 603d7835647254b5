// Small device utilities of libvp: prefix sums, reductions, pair split.
#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>

#include "vp_internal.h"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Inclusive scan of one tile per block into out[i]; block totals to sums[b].
template <typename T>
__global__ void k_scan_tile(const T* __restrict__ in, int64_t* __restrict__ out, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t run = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        run += (idx < n) ? (int64_t)in[idx] : 0;
        v[i] = run;
    }
    // exclusive scan of per-thread totals across the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    int64_t prefix = x - run + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = v[i] + prefix;
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = prefix + run;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int64_t b = i / SCAN_TILE;
        if (b > 0) out[i] += offs[b - 1];
    }
}

__global__ void k_zero_first(int64_t* out) { out[0] = 0; }

template <typename T>
int scan_inclusive(vp_ctx* ctx, const T* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return VP_OK;
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t* sums = nullptr;
    VP_CUDA_TRY(ctx, cudaMallocAsync(&sums, nb * sizeof(int64_t), s));
    k_scan_tile<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    VP_LAUNCH_CHECK(ctx);
    if (nb > 1) {
        int64_t* sums2 = nullptr;
        VP_CUDA_TRY(ctx, cudaMallocAsync(&sums2, nb * sizeof(int64_t), s));
        int rc = scan_inclusive<int64_t>(ctx, sums, sums2, nb, s);
        if (rc) return rc;
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums2);
        VP_LAUNCH_CHECK(ctx);
        VP_CUDA_TRY(ctx, cudaFreeAsync(sums2, s));
    }
    VP_CUDA_TRY(ctx, cudaFreeAsync(sums, s));
    return VP_OK;
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, int32_t* out) {
    int32_t m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_sum_i32(const int32_t* __restrict__ a, int64_t n, unsigned long long* out) {
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m += (unsigned long long)(uint32_t)a[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, m);
}

// out[0] += sum of a over kind 0, out[1] += over kind != 0, out[2] += sum of b
__global__ void k_sum_by_kind(const int32_t* __restrict__ a, const uint8_t* __restrict__ kind,
                              const int32_t* __restrict__ b, int64_t n, unsigned long long* out) {
    unsigned long long s0 = 0, s1 = 0, sb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long v = (uint32_t)a[i];
        if (kind[i]) s1 += v;
        else s0 += v;
        sb += (uint32_t)b[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], s0);
        atomicAdd(&out[1], s1);
        atomicAdd(&out[2], sb);
    }
}

// Compact pair indices by kind (order within each list is irrelevant: every
// pair writes only its own output row).
__global__ void k_split_pairs(const uint8_t* __restrict__ kind, int64_t P, int32_t* near_idx, int32_t* self_idx,
                              unsigned long long* counters) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < P;
    bool is_self = valid && kind[i] == 1;
    bool is_near = valid && kind[i] == 0;
    unsigned ms = __ballot_sync(0xffffffffu, is_self);
    unsigned mn = __ballot_sync(0xffffffffu, is_near);
    int lane = threadIdx.x & 31;
    unsigned long long bs = 0, bn = 0;
    if (lane == 0) {
        if (ms) bs = atomicAdd(&counters[1], (unsigned long long)__popc(ms));
        if (mn) bn = atomicAdd(&counters[0], (unsigned long long)__popc(mn));
    }
    bs = __shfl_sync(0xffffffffu, bs, 0);
    bn = __shfl_sync(0xffffffffu, bn, 0);
    unsigned lower = (1u << lane) - 1u;
    if (is_self) self_idx[bs + __popc(ms & lower)] = (int32_t)i;
    if (is_near) near_idx[bn + __popc(mn & lower)] = (int32_t)i;
}

}  // namespace

int vp_exclusive_scan_i32(vp_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    k_zero_first<<<1, 1, 0, s>>>(out);
    VP_LAUNCH_CHECK(ctx);
    return scan_inclusive<int32_t>(ctx, in, out + 1, n, s);
}

int vp_exclusive_scan_i64(vp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    k_zero_first<<<1, 1, 0, s>>>(out);
    VP_LAUNCH_CHECK(ctx);
    return scan_inclusive<int64_t>(ctx, in, out + 1, n, s);
}

void launch_max_i32(const int32_t* a, int64_t n, int32_t* out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    if (n > 0) k_max_i32<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(a, n, out);
}

void launch_sum_i32(const int32_t* a, int64_t n, unsigned long long* out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (n > 0) k_sum_i32<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(a, n, out);
}

void launch_sum_by_kind(const int32_t* a, const uint8_t* kind, const int32_t* b, int64_t n, unsigned long long* out,
                        cudaStream_t s) {
    cudaMemsetAsync(out, 0, 3 * sizeof(unsigned long long), s);
    if (n > 0) k_sum_by_kind<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(a, kind, b, n, out);
}

void launch_split_pairs(const uint8_t* pkind, int64_t P, int32_t* near_idx, int32_t* self_idx,
                        unsigned long long* counters, cudaStream_t s) {
    cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), s);
    if (P > 0) k_split_pairs<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(pkind, P, near_idx, self_idx, counters);
}
