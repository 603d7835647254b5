// Correction apply of one density in the mixed path, streamed through shared
// memory by the bulk-copy engine: the last sum of the subtract-and-add
// evaluation (Section 3.6),
//     u(x_t) += sum_{(t, T) in lists} sum_k C[t,T,k] f_{T,k}.
//
// The weights are pair-major (pairs in target order, nq float-float weights
// per pair), so a run of pairs is a run of bytes.  Work is cut into tiles of
// 32 pairs (4,864 bytes of weights for nq = 19).  Each warp of a persistent
// grid owns a ring of VP_AS_STAGES tiles in shared memory that one lane
// refills with cp.async.bulk (three copies per tile: weights, triangles,
// targets, all completing on the stage's mbarrier), so that the warp computes
// one tile while the next ones stream in.  Lane l takes pair p0 + l: its
// weights from the tile, its triangle's density values from the L2-resident
// float-float density, padded to fd2_stride(nq) pairs per triangle so that
// they come in 16-byte loads (half the gather instructions of 8-byte ones),
// the products split exactly into four float-float partial sums; then a
// float-float segmented sum over the lanes by target (the pairs of a target
// are adjacent).  The FP64 pipe, slow on this part, only converts the segment
// sums.  A target whose whole row lies in the tile (read off the targets of
// the pairs just before and after the tile) gets its one update as an atomic
// add; the first and last segment of a tile whose rows cross the tile
// boundary go to two per-tile slots, and a second kernel adds those, in tile
// order, to the targets whose rows cross tiles.  The order of every sum is
// fixed, so the result does not depend on timing.
#include <algorithm>
#include <climits>

#include "vp_internal.h"
#include "vp_async.cuh"
#include "vp_f2.cuh"

#ifndef VP_AS_WARPS
#define VP_AS_WARPS 22
#endif
#ifndef VP_AS_STAGES
#define VP_AS_STAGES 2
#endif

namespace {

constexpr int AS_WARPS = VP_AS_WARPS;
constexpr int AS_STAGES = VP_AS_STAGES;
constexpr int AS_TILE = 32;   // pairs per tile, one per lane

template <int NQ>
struct __align__(16) AsStage {
    float2 C[AS_TILE * NQ];   // weights of the tile's pairs, (h, l) per weight
    int32_t tri[AS_TILE];     // triangle of each pair
    int32_t tgt[AS_TILE];     // target of each pair
};

template <int NQ>
constexpr size_t as_smem_bytes() {
    return (size_t)AS_WARPS * AS_STAGES * sizeof(AsStage<NQ>) + (size_t)AS_WARPS * AS_STAGES * sizeof(uint64_t);
}

template <int NQ>
__global__ void __launch_bounds__(AS_WARPS * 32, 1)
    k_apply_stream(const int32_t* __restrict__ ptri, const int32_t* __restrict__ ptgt,
                   const float2* __restrict__ C2, const float2* __restrict__ fd2, int64_t P, double* __restrict__ u,
                   double* __restrict__ slots, int32_t* flag) {
    extern __shared__ __align__(128) unsigned char smem[];
    using St = AsStage<NQ>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    St* st = reinterpret_cast<St*>(smem) + wid * AS_STAGES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + AS_WARPS * AS_STAGES * sizeof(St)) + wid * AS_STAGES;
    const int64_t ntiles = (P + AS_TILE - 1) / AS_TILE;
    const int64_t stride = (int64_t)gridDim.x * AS_WARPS;
    const int64_t first = (int64_t)blockIdx.x * AS_WARPS + wid;
    if (lane == 0) {
        for (int s = 0; s < AS_STAGES; s++) mbar_init(smem_u32(&bar[s]), 1);
        fence_mbar_init();
    }
    __syncwarp();
    // one lane: stream tile `tile` into stage s (sizes rounded up to 16 bytes;
    // the arrays carry 16 bytes of padding past their last element)
    auto issue = [&](int s, int64_t tile) {
        const int64_t p0 = tile * AS_TILE;
        const int n = (int)min((int64_t)AS_TILE, P - p0);
        const uint32_t cb = (uint32_t)((n * NQ * (int)sizeof(float2) + 15) & ~15);
        const uint32_t ib = (uint32_t)((n * (int)sizeof(int32_t) + 15) & ~15);
        const uint32_t b = smem_u32(&bar[s]);
        mbar_expect_tx(b, cb + 2 * ib);
        bulk_g2s(smem_u32(st[s].C), C2 + p0 * NQ, cb, b);
        bulk_g2s(smem_u32(st[s].tri), ptri + p0, ib, b);
        bulk_g2s(smem_u32(st[s].tgt), ptgt + p0, ib, b);
    };
    if (lane == 0)
        for (int s = 0; s < AS_STAGES; s++)
            if (first + s * stride < ntiles) issue(s, first + s * stride);
    int64_t k = 0;
    bool ok = true;
    for (int64_t tile = first; tile < ntiles; tile += stride, k++) {
        const int s = (int)(k % AS_STAGES);
        if (!mbar_wait(smem_u32(&bar[s]), (uint32_t)((k / AS_STAGES) & 1))) {
            ok = false;
            break;
        }
        const int64_t p0 = tile * AS_TILE;
        const int n = (int)min((int64_t)AS_TILE, P - p0);
        // pair-parallel: lane l takes pair p0 + l.  Its weights come from the
        // tile in shared memory, its density values straight from the
        // L2-resident float-float density (one triangle's values contiguous);
        // each product is split exactly and added into one of four
        // float-float partial sums (hi by two-sum, lo collecting the errors)
        // in a fixed order.
        const int pl = lane;
        int t = INT_MAX;   // padding lanes form their own segment
        // the targets of the pairs just before and just after the tile (-1
        // past either end): whether a row crosses the tile's edges
        int nb = -1;
        if (lane == 0 && p0 > 0) nb = __ldg(ptgt + p0 - 1);
        if (lane == 1 && p0 + n < P) nb = __ldg(ptgt + p0 + n);
        f2 ps = {0.f, 0.f};
        if (pl < n) {
            t = st[s].tgt[pl];
            // the triangle's values, fd2_stride(NQ) pairs from a 16-byte boundary: 16-byte loads
            const float4* fp = reinterpret_cast<const float4*>(fd2 + (int64_t)st[s].tri[pl] * fd2_stride(NQ));
            float2 fv[NQ + 1];
#pragma unroll
            for (int q = 0; q < (NQ + 1) / 2; q++) {
                const float4 v4 = __ldg(fp + q);
                fv[2 * q] = make_float2(v4.x, v4.y);
                fv[2 * q + 1] = make_float2(v4.z, v4.w);
            }
            const float2* c = st[s].C + pl * NQ;
            float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                const float2 cv = c[q];
                f2_acc(ah[q & 3], al[q & 3], f2{cv.x, cv.y}, f2{fv[q].x, fv[q].y});
            }
            ps = f2_add(f2_add(f2_fast(ah[0], al[0]), f2_fast(ah[1], al[1])),
                        f2_add(f2_fast(ah[2], al[2]), f2_fast(ah[3], al[3])));
        }
        // segmented inclusive sum over the pairs (targets are non-decreasing)
#pragma unroll
        for (int o = 1; o < AS_TILE; o <<= 1) {
            const float vh = __shfl_up_sync(0xffffffffu, ps.h, o, AS_TILE);
            const float vl = __shfl_up_sync(0xffffffffu, ps.l, o, AS_TILE);
            const int kt = __shfl_up_sync(0xffffffffu, t, o, AS_TILE);
            if (pl >= o && kt == t) ps = f2_add(ps, {vh, vl});
        }
        const int t_next = __shfl_down_sync(0xffffffffu, t, 1, AS_TILE);
        const int t_lane0 = __shfl_sync(0xffffffffu, t, 0);
        const int t_before = __shfl_sync(0xffffffffu, nb, 0), t_after = __shfl_sync(0xffffffffu, nb, 1);
        if (lane == pl && lane < n && (lane == n - 1 || t_next != t)) {   // the last pair of a segment
            const double sum = (double)ps.h + (double)ps.l;
            const bool starts_here = !(t == t_lane0 && t_before == t), ends_here = !(lane == n - 1 && t_after == t);
            if (starts_here && ends_here) {
                atomicAdd(u + t, sum);                        // the whole row is in this tile: its only update
            } else {
                if (t == t_lane0) slots[2 * tile] = sum;      // segment at the start of the tile
                if (lane == n - 1) slots[2 * tile + 1] = sum; // segment at the end of the tile
            }
        }
        __syncwarp();
        if (lane == 0 && tile + AS_STAGES * stride < ntiles) issue(s, tile + AS_STAGES * stride);
    }
    if (!ok) {
        // a copy never completed: report, wait (bounded) for the copies still
        // in flight into this warp's stages, and leave
        if (lane == 0) {
            atomicOr(flag, VP_DEV_ERR_TIMEOUT);
            for (int j = 0; j < AS_STAGES; j++) {
                const int64_t kk = k + j;
                if (first + kk * stride < ntiles)
                    mbar_wait(smem_u32(&bar[kk % AS_STAGES]), (uint32_t)((kk / AS_STAGES) & 1));
            }
        }
        __syncwarp();
    }
}

// Targets whose rows cross tiles: u[t] += (end segment of the first tile) +
// (whole middle tiles) + (start segment of the last tile), in tile order.
__global__ void k_apply_stream_fix(const int64_t* __restrict__ row, int64_t M, const double* __restrict__ slots,
                                   double* __restrict__ u) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    const int64_t r0 = row[t], r1 = row[t + 1];
    if (r1 <= r0) return;
    const int64_t a = r0 / AS_TILE, b = (r1 - 1) / AS_TILE;
    if (a == b) return;
    double s = slots[2 * a + 1];
    for (int64_t i = a + 1; i < b; i++) s += slots[2 * i];
    s += slots[2 * b];
    u[t] += s;
}

template <int NQ>
void apply_stream(const int64_t* row, const int32_t* ptri, const int32_t* ptgt, const float2* C2, const float2* fd2,
                  int64_t P, int64_t M, double* u, double* slots, int32_t* flag, int sm_count, cudaStream_t s) {
    constexpr size_t smem = as_smem_bytes<NQ>();
    // the shared-memory attribute once per device (not again inside a graph capture)
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(k_apply_stream<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const int64_t ntiles = (P + AS_TILE - 1) / AS_TILE;
    // one CTA per SM (persistent), fewer when there are fewer tiles than warps
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(sm_count, (ntiles + AS_WARPS - 1) / AS_WARPS));
    k_apply_stream<NQ><<<grid, AS_WARPS * 32, smem, s>>>(ptri, ptgt, C2, fd2, P, u, slots, flag);
    k_apply_stream_fix<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(row, M, slots, u);
}

}  // namespace

// the padded float-float density: at most N (nq + 1) / nq <= N 17/16 pairs
// for nq >= 16
static size_t fd2_region_bytes(int64_t N) {
    return ((size_t)(N + N / 16 + 2) * sizeof(float2) + 255) & ~(size_t)255;
}

size_t apply_stream_ws_bytes(int64_t N, int64_t P) {
    return fd2_region_bytes(N) + (size_t)((P + AS_TILE - 1) / AS_TILE) * 2 * sizeof(double);
}

// f (node values, FP64) -> the padded triangle-major float-float density
__global__ void k_to_fd2(const double* __restrict__ f, int64_t N, int nq, float2* __restrict__ fd2) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double v = f[j];
    const float h = __double2float_rn(v);
    fd2[(j / nq) * fd2_stride(nq) + j % nq] = make_float2(h, __double2float_rn(v - (double)h));
}

void launch_apply_stream(const int64_t* row, const int32_t* ptri, const int32_t* ptgt, const float2* C2, int nq,
                         const double* f, int64_t N, int64_t P, int64_t M, double* u, void* ws, int32_t* flag,
                         int sm_count, cudaStream_t s, bool f2_ready) {
    if (P <= 0 || M <= 0) return;
    // the density as float-float pairs, then the slots
    float2* fd2 = (float2*)ws;
    double* slots = (double*)((char*)ws + fd2_region_bytes(N));
    if (!f2_ready) k_to_fd2<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(f, N, nq, fd2);
    if (nq == 19) apply_stream<19>(row, ptri, ptgt, C2, fd2, P, M, u, slots, flag, sm_count, s);
    else apply_stream<16>(row, ptri, ptgt, C2, fd2, P, M, u, slots, flag, sm_count, s);
}
