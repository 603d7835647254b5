// Batched evaluation of many near-field builds (possibly different meshes and
// density counts): one persistent far-sum launch per density-chunk width over
// all items, one correction launch over all items' targets, captured once in
// a CUDA graph and replayed.  Work units of the far sum are (item, block of
// target rows) taken from an atomic counter, so uneven meshes balance.
// Results agree with vp_potential_eval item by item up to the order of the
// far-sum partial sums (vp_potential_eval may split the sources of small
// target sets over several blocks; here every unit sums all its sources).
#include <algorithm>
#include <new>
#include <vector>

#include "vp_internal.h"
#include "vp_ff.cuh"

namespace {

struct BatchFar {
    const float* shi;
    const float* slo;
    const float* q;
    int64_t N;
    const float* thi;
    const float* tlo;
    const int32_t* tnode;
    int64_t M;
    double* u;
    int d, d0;
    int64_t unit_begin;    // first work unit of this entry
    int64_t units;         // target blocks of this entry
};

struct BatchApply {
    const int64_t* row;
    const int32_t* ptri;
    const double* C;
    const double* f;
    double* u;
    int64_t N, M;
    int nq, d;
    int64_t t_begin;       // first global target of this item
};

__device__ __forceinline__ int find_entry(const int64_t* begins, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begins[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int D, int TPT>
__global__ void __launch_bounds__(FF_THREADS) k_far_ff_batch(const BatchFar* __restrict__ ent,
                                                             const int64_t* __restrict__ begins, int nent,
                                                             int64_t total_units, unsigned long long* counter) {
    __shared__ FFSmem<D> sm;
    __shared__ long long unit_s;
    ff_load_table(sm);
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) unit_s = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t unit = unit_s;
        if (unit >= total_units) break;
        const int e = find_entry(begins, nent, unit);
        const BatchFar& E = ent[e];
        const int64_t b = unit - E.unit_begin;
        const int64_t tbase = b * (FF_THREADS * TPT) + threadIdx.x;
        ff_far_block<D, TPT>(sm, E.shi, E.slo, E.q, 0, E.N, E.thi, E.tlo, E.tnode, E.M, tbase, E.d, E.d0, E.u);
    }
}

// Warp per global target over all items: u[k][t] += sum_e C[e] f[k][T_e nq + node].
__global__ void k_apply_batch(const BatchApply* __restrict__ it, const int64_t* __restrict__ begins, int n,
                              int64_t total) {
    const int lane = threadIdx.x & 31;
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= total) return;
    const int i = find_entry(begins, n, g);
    const BatchApply& A = it[i];
    const int64_t t = g - A.t_begin;
    const int nq = A.nq;
    const int64_t e0 = A.row[t] * nq, e1 = A.row[t + 1] * nq;
    for (int k = 0; k < A.d; k++) {
        const double* fk = A.f + (int64_t)k * A.N;
        double s = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t p = e / nq;
            const int node = (int)(e - p * nq);
            s += A.C[e] * fk[(int64_t)A.ptri[p] * nq + node];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) A.u[(int64_t)k * A.M + t] += s;
    }
}

template <int D, int TPT>
void launch_batch_far(const BatchFar* ent, const int64_t* begins, int nent, int64_t units, unsigned long long* counter,
                      int grid, cudaStream_t s) {
    k_far_ff_batch<D, TPT><<<grid, FF_THREADS, 0, s>>>(ent, begins, nent, units, counter);
}

typedef void (*BatchFarFn)(const BatchFar*, const int64_t*, int, int64_t, unsigned long long*, int, cudaStream_t);

template <int D>
BatchFarFn far_fn(int tpt) {
    switch (tpt) {
        case 1: return launch_batch_far<D, 1>;
        case 4: return launch_batch_far<D, 4>;
        default: return launch_batch_far<D, 2>;
    }
}

BatchFarFn far_fn_d(int D, int tpt) {
    switch (D) {
        case 8: return far_fn<8>(tpt);
        case 4: return far_fn<4>(tpt);
        case 2: return far_fn<2>(tpt);
        default: return far_fn<1>(tpt);
    }
}

template <int D, int TPT>
int occupancy_of() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_far_ff_batch<D, TPT>, FF_THREADS, 0);
    return std::max(1, nb);
}

int occupancy(int D, int tpt) {
    switch (D * 8 + tpt) {
        case 8 * 8 + 1: return occupancy_of<8, 1>();
        case 8 * 8 + 2: return occupancy_of<8, 2>();
        case 8 * 8 + 4: return occupancy_of<8, 4>();
        case 4 * 8 + 1: return occupancy_of<4, 1>();
        case 4 * 8 + 2: return occupancy_of<4, 2>();
        case 4 * 8 + 4: return occupancy_of<4, 4>();
        case 2 * 8 + 1: return occupancy_of<2, 1>();
        case 2 * 8 + 2: return occupancy_of<2, 2>();
        case 2 * 8 + 4: return occupancy_of<2, 4>();
        case 1 * 8 + 1: return occupancy_of<1, 1>();
        case 1 * 8 + 4: return occupancy_of<1, 4>();
        default: return occupancy_of<1, 2>();
    }
}

struct DevGuardB {
    int prev = -1;
    explicit DevGuardB(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuardB() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int chunk_width(int rest) { return rest >= 8 ? 8 : (rest >= 4 ? 4 : (rest >= 2 ? 2 : 1)); }
int group_of(int D) { return D == 8 ? 3 : (D == 4 ? 2 : (D == 2 ? 1 : 0)); }

}  // namespace

struct vp_batch {
    vp_ctx* ctx = nullptr;
    int precision = 0;
    std::vector<vp_eval_item> items;
    // per density-chunk group (D = 1, 2, 4, 8)
    BatchFar* d_far[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t* d_far_begin[4] = {nullptr, nullptr, nullptr, nullptr};
    int nent[4] = {0, 0, 0, 0};
    int64_t units[4] = {0, 0, 0, 0};
    int tpt[4] = {2, 2, 2, 2};
    int grid[4] = {0, 0, 0, 0};
    BatchApply* d_apply = nullptr;
    int64_t* d_apply_begin = nullptr;
    int64_t total_targets = 0;
    float* qbuf = nullptr;
    unsigned long long* counters = nullptr;
    // per (item, chunk): charge preparation
    struct Prep {
        const double* W;
        const double* f;
        int64_t N;
        int d, d0, D;
        float* q;
    };
    std::vector<Prep> preps;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* fmm_ws = nullptr;        // VP_MIXED_FMM: one workspace, items run in turn
    int magic = 0x56504254;
};

static void enqueue(vp_batch* b, cudaStream_t s) {
    vp_ctx* ctx = b->ctx;
    if (b->precision == VP_MIXED) {
        cudaMemsetAsync(b->counters, 0, 4 * sizeof(unsigned long long), s);
        for (const auto& p : b->preps) {
            const unsigned pb = (unsigned)((p.N + 255) / 256);
            switch (p.D) {
                case 8: k_prep_q_ff<8><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                case 4: k_prep_q_ff<4><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                case 2: k_prep_q_ff<2><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                default: k_prep_q_ff<1><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
            }
        }
        for (int g = 0; g < 4; g++) {
            if (!b->nent[g]) continue;
            const int D = 1 << g;
            far_fn_d(D, b->tpt[g])(b->d_far[g], b->d_far_begin[g], b->nent[g], b->units[g], b->counters + g,
                                   b->grid[g], s);
        }
    } else {
        for (const auto& it : b->items)
            launch_far_fp64(it.nf->mesh->d_y, it.nf->mesh->d_W, it.nf->mesh->N, it.f_dev, it.d, it.nf->d_txy,
                            it.nf->d_tnode, it.nf->M, it.u_dev, 1, s);
    }
    const int64_t total = b->total_targets;
    if (total > 0)
        k_apply_batch<<<(unsigned)((total * 32 + 255) / 256), 256, 0, s>>>(b->d_apply, b->d_apply_begin,
                                                                        (int)b->items.size(), total);
    (void)ctx;
}

static void free_batch(vp_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int g = 0; g < 4; g++) {
        if (b->d_far[g]) cudaFree(b->d_far[g]);
        if (b->d_far_begin[g]) cudaFree(b->d_far_begin[g]);
    }
    if (b->d_apply) cudaFree(b->d_apply);
    if (b->d_apply_begin) cudaFree(b->d_apply_begin);
    if (b->qbuf) cudaFree(b->qbuf);
    if (b->counters) cudaFree(b->counters);
    if (b->fmm_ws) cudaFree(b->fmm_ws);
    b->magic = 0;
    delete b;
}

// VP_MIXED_FMM batches: the multipole plans of the items (built here when
// missing), one workspace for the largest item, and every item's evaluation
// (multipole far sum, then the corrections) captured in turn into one graph.
static int batch_create_fmm(vp_ctx* ctx, vp_batch* b, cudaStream_t s) {
    size_t ws = 0;
    for (const auto& it : b->items) {
        vp_nf* nf = const_cast<vp_nf*>(it.nf);
        if (!nf->fmm) {
            const int rc = fmm_plan_build(ctx, nf, s);
            if (rc) return rc;
        }
        ws = std::max(ws, eval_ws_bytes(ctx, nf, it.d, VP_MIXED_FMM));
    }
    if (cudaMalloc(&b->fmm_ws, std::max<size_t>(ws, 256)) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_OOM, "vp_batch_create: workspace");
    // one evaluation outside the capture (first-use set-up of the kernels)
    const vp_eval_item& i0 = b->items[0];
    int rc = eval_impl(ctx, i0.nf, i0.f_dev, i0.d, i0.u_dev, VP_MIXED_FMM, s, b->fmm_ws, false);
    if (rc) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return vp_set_error(ctx, VP_ERR_CUDA, "vp_batch_create: warm-up");
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_CUDA, "vp_batch_create: stream");
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_CUDA, "vp_batch_create: capture");
    for (const auto& it : b->items) {
        rc = eval_impl(ctx, it.nf, it.f_dev, it.d, it.u_dev, VP_MIXED_FMM, b->cap, b->fmm_ws, false);
        if (rc) break;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
    b->graph = g;
    if (rc) return rc;
    if (ec != cudaSuccess || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_CUDA, "vp_batch_create: graph");
    b->total_targets = 0;
    for (const auto& it : b->items) b->total_targets += it.nf->M;
    return VP_OK;
}

extern "C" int vp_batch_create(vp_ctx* ctx, const vp_eval_item* items, int32_t n, int32_t precision, void* stream,
                               vp_batch** out) {
    if (out) *out = nullptr;
    if (!ctx || ctx->magic != 0x56504358) return VP_ERR_STATE;
    if (!out || n < 1 || !items || (precision != VP_FP64 && precision != VP_MIXED && precision != VP_MIXED_FMM))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_batch_create: bad arguments");
    for (int32_t i = 0; i < n; i++) {
        const vp_eval_item& it = items[i];
        if (!it.nf || it.nf->magic != 0x56504e46 || it.nf->ctx != ctx)
            return vp_set_error(ctx, VP_ERR_STATE, "vp_batch_create: bad near-field handle");
        if (!it.f_dev || !it.u_dev || it.d < 1 || it.d > 256)
            return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_batch_create: bad item");
    }
    DevGuardB guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    vp_batch* b = new (std::nothrow) vp_batch();
    if (!b) return VP_ERR_OOM;
    b->ctx = ctx;
    b->precision = precision;
    b->items.assign(items, items + n);
    int rc = VP_OK;
    if (precision == VP_MIXED_FMM) {
        rc = batch_create_fmm(ctx, b, s);
        if (rc) {
            free_batch(b);
            return rc;
        }
        *out = b;
        return VP_OK;
    }
    // far-sum entries per chunk width, charge buffers, apply descriptors
    std::vector<BatchFar> far[4];
    std::vector<int64_t> far_begin[4];
    std::vector<BatchApply> app;
    std::vector<int64_t> app_begin;
    size_t qfloats = 0;
    for (const auto& it : b->items)
        for (int d0 = 0; d0 < it.d;) {
            const int D = chunk_width(it.d - d0);
            qfloats += (size_t)it.nf->mesh->N * 2 * D;
            d0 += D;
        }
    if (precision == VP_MIXED && cudaMalloc(&b->qbuf, std::max<size_t>(qfloats, 1) * sizeof(float)) != cudaSuccess) {
        free_batch(b);
        return vp_set_error(ctx, VP_ERR_OOM, "vp_batch_create: charge buffer");
    }
    size_t qoff = 0;
    for (const auto& it : b->items) {
        const vp_nf* nf = it.nf;
        const vp_mesh* mesh = nf->mesh;
        for (int d0 = 0; d0 < it.d;) {
            const int D = chunk_width(it.d - d0);
            const int g = group_of(D);
            float* q = b->qbuf ? b->qbuf + qoff : nullptr;
            qoff += (size_t)mesh->N * 2 * D;
            b->preps.push_back({mesh->d_W, it.f_dev, mesh->N, it.d, d0, D, q});
            BatchFar e;
            e.shi = nf->src_ff.hi;
            e.slo = nf->src_ff.lo;
            e.q = q;
            e.N = mesh->N;
            e.thi = nf->tgt_ff.hi;
            e.tlo = nf->tgt_ff.lo;
            e.tnode = nf->d_tnode;
            e.M = nf->M;
            e.u = it.u_dev;
            e.d = it.d;
            e.d0 = d0;
            e.unit_begin = 0;
            e.units = 0;
            far[g].push_back(e);
            d0 += D;
        }
        BatchApply a;
        a.row = nf->d_row;
        a.ptri = nf->d_ptri;
        a.C = nf->d_C;
        a.f = it.f_dev;
        a.u = it.u_dev;
        a.N = mesh->N;
        a.M = nf->M;
        a.nq = mesh->nq;
        a.d = it.d;
        a.t_begin = b->total_targets;
        app.push_back(a);
        app_begin.push_back(b->total_targets);
        b->total_targets += nf->M;
    }
    auto upload = [&](void** dst, const void* src, size_t bytes) -> bool {
        if (cudaMalloc(dst, std::max<size_t>(bytes, 1)) != cudaSuccess) return false;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (cudaMalloc(&b->counters, 4 * sizeof(unsigned long long)) != cudaSuccess) rc = VP_ERR_OOM;
    // tile shape per chunk width: the project's autotuner times each
    // targets-per-thread variant once per context and keeps the fastest
    for (int g = 0; g < 4 && rc == VP_OK; g++) {
        if (far[g].empty()) continue;
        const int D = 1 << g;
        b->nent[g] = (int)far[g].size();
        const int fixed = ctx->ff_tpt_fixed[g];
        b->tpt[g] = fixed ? fixed : (ctx->ff_tpt[g] ? ctx->ff_tpt[g] : 2);
        auto fill_units = [&](int tpt) {
            int64_t u = 0;
            for (size_t i = 0; i < far[g].size(); i++) {
                far[g][i].unit_begin = u;
                far[g][i].units = (far[g][i].M + FF_THREADS * tpt - 1) / (FF_THREADS * tpt);
                far_begin[g].push_back(u);
                u += far[g][i].units;
            }
            b->units[g] = u;
        };
        fill_units(b->tpt[g]);
        if (!upload((void**)&b->d_far[g], far[g].data(), far[g].size() * sizeof(BatchFar)) ||
            !upload((void**)&b->d_far_begin[g], far_begin[g].data(), far_begin[g].size() * sizeof(int64_t)))
            rc = VP_ERR_OOM;
        b->grid[g] = ctx->sm_count * occupancy(D, b->tpt[g]);
        if (rc == VP_OK && !fixed && !ctx->ff_tpt[g] && precision == VP_MIXED) {
            // autotune on this batch: charges first, then each variant timed
            for (const auto& p : b->preps)
                if (p.D == D) {
                    const unsigned pb = (unsigned)((p.N + 255) / 256);
                    switch (D) {
                        case 8: k_prep_q_ff<8><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                        case 4: k_prep_q_ff<4><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                        case 2: k_prep_q_ff<2><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                        default: k_prep_q_ff<1><<<pb, 256, 0, s>>>(p.W, p.f, p.N, p.d, p.d0, p.q); break;
                    }
                }
            float best = 1e30f;
            int best_tpt = 2;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            // time on the leading entries only, up to about 2e10 source-target pairs
            int ntune = 0;
            double pairs = 0.0;
            while (ntune < b->nent[g] && (ntune == 0 || pairs < 2e10)) {
                pairs += (double)far[g][ntune].N * (double)far[g][ntune].M;
                ntune++;
            }
            for (int tpt : {1, 2, 4}) {
                far_begin[g].clear();
                fill_units(tpt);
                cudaMemcpy(b->d_far[g], far[g].data(), far[g].size() * sizeof(BatchFar), cudaMemcpyHostToDevice);
                cudaMemcpy(b->d_far_begin[g], far_begin[g].data(), far_begin[g].size() * sizeof(int64_t),
                           cudaMemcpyHostToDevice);
                const int grid = ctx->sm_count * occupancy(D, tpt);
                const int64_t tune_units = ntune < b->nent[g] ? far_begin[g][ntune] : b->units[g];
                cudaMemsetAsync(b->counters + g, 0, sizeof(unsigned long long), s);
                cudaEventRecord(e0, s);
                far_fn_d(D, tpt)(b->d_far[g], b->d_far_begin[g], ntune, tune_units, b->counters + g, grid, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_tpt = tpt;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ctx->ff_tpt[g] = best_tpt;
            b->tpt[g] = best_tpt;
            far_begin[g].clear();
            fill_units(best_tpt);
            cudaMemcpy(b->d_far[g], far[g].data(), far[g].size() * sizeof(BatchFar), cudaMemcpyHostToDevice);
            cudaMemcpy(b->d_far_begin[g], far_begin[g].data(), far_begin[g].size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice);
            b->grid[g] = ctx->sm_count * occupancy(D, best_tpt);
        }
    }
    if (rc == VP_OK && (!upload((void**)&b->d_apply, app.data(), app.size() * sizeof(BatchApply)) ||
                        !upload((void**)&b->d_apply_begin, app_begin.data(), app_begin.size() * sizeof(int64_t))))
        rc = VP_ERR_OOM;
    if (rc == VP_OK) ensure_logtab();
    // capture the launch sequence once; replays re-read the items' densities
    if (rc == VP_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) rc = VP_ERR_CUDA;
    if (rc == VP_OK) {
        cudaStreamSynchronize(s);
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = VP_ERR_CUDA;
        else {
            enqueue(b, b->cap);
            if (cudaStreamEndCapture(b->cap, &b->graph) != cudaSuccess ||
                cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
                rc = VP_ERR_CUDA;
        }
    }
    if (rc != VP_OK) {
        cudaError_t le = cudaGetLastError();
        free_batch(b);
        return vp_set_error(ctx, rc, std::string("vp_batch_create: ") + cudaGetErrorString(le));
    }
    *out = b;
    return VP_OK;
}

extern "C" int vp_set_batch_tile(vp_ctx* ctx, int32_t width, int32_t targets_per_thread) {
    if (!ctx || ctx->magic != 0x56504358) return VP_ERR_STATE;
    const int g = width == 1 ? 0 : width == 2 ? 1 : width == 4 ? 2 : width == 8 ? 3 : -1;
    if (g < 0 || (targets_per_thread != 0 && targets_per_thread != 1 && targets_per_thread != 2 &&
                  targets_per_thread != 4))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_set_batch_tile: width 1/2/4/8, targets per thread 0/1/2/4");
    ctx->ff_tpt_fixed[g] = targets_per_thread;
    return VP_OK;
}

extern "C" int vp_batch_info(const vp_batch* b, int32_t* targets_per_thread, int64_t* work_units) {
    if (!b || b->magic != 0x56504254) return VP_ERR_STATE;
    for (int g = 0; g < 4; g++) {
        const bool used = b->nent[g] > 0 && b->precision != VP_MIXED_FMM;
        if (targets_per_thread) targets_per_thread[g] = used ? b->tpt[g] : 0;
        if (work_units) work_units[g] = used ? b->units[g] : 0;
    }
    return VP_OK;
}

extern "C" int vp_batch_launch(vp_batch* b, void* stream) {
    if (!b || b->magic != 0x56504254) return VP_ERR_STATE;
    DevGuardB guard(b->ctx->device);
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return vp_set_error(b->ctx, VP_ERR_CUDA, std::string("vp_batch_launch: ") + cudaGetErrorString(e));
    return VP_OK;
}

extern "C" void vp_batch_release(vp_batch* b) {
    if (!b || b->magic != 0x56504254) return;
    DevGuardB guard(b->ctx->device);
    cudaDeviceSynchronize();
    free_batch(b);
}

extern "C" int vp_potential_eval_batch(vp_ctx* ctx, const vp_eval_item* items, int32_t n, int32_t precision,
                                       void* stream) {
    if (!ctx || ctx->magic != 0x56504358) return VP_ERR_STATE;
    if (n == 0) return VP_OK;
    vp_batch* b = nullptr;
    int rc = vp_batch_create(ctx, items, n, precision, stream, &b);
    if (rc) return rc;
    rc = vp_batch_launch(b, stream);
    if (rc == VP_OK) cudaStreamSynchronize((cudaStream_t)stream);
    vp_batch_release(b);
    return rc;
}

// Loads this unit's log table on the current device (vp_create).
cudaError_t batch_module_prepare() { return ensure_logtab(); }
