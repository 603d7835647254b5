// vp_potential_eval_noalloc: the potential evaluation with its far-sum
// scratch in a fixed device array instead of memory allocated at run time.
//
// Some callers cannot allocate device memory while they evaluate: a process
// whose GPU memory is already owned by another allocator (a caching
// allocator such as PyTorch's can hold every free byte, so cudaMalloc fails
// although the caller has room in its own pool), or a latency-bound serving
// loop that cannot accept the device-wide synchronisation cudaMalloc and
// cudaFree perform.  This entry point runs the same kernels as
// vp_potential_eval but takes its scratch (split-source partial sums and the
// float-float charges) from g_eval_scratch below and calls no allocator.
#include <mutex>

#include "vp_internal.h"

namespace {

// Fixed scratch of the allocation-free evaluation.  Every GPU that loads the
// library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_eval_scratch[kScratchBytes];

// The array's device address, looked up once per device (host code must not
// use the symbol's name as an address).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~CurrentDevice() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Called with ctx->device current (vp_create, then every call: a lookup).
int scratch_address(vp_ctx* ctx, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const int dev = ctx->device;
    if (dev < 0 || dev >= kMaxDevices)
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_potential_eval_noalloc: device index above 63");
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_eval_scratch);
        if (e != cudaSuccess || !p)
            return vp_set_error(ctx, VP_ERR_CUDA,
                                std::string("vp_potential_eval_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_addr[dev];
    return VP_OK;
}

}  // namespace

// Run by vp_create with the device current: resolving the address loads this
// unit's module, which reserves the array, so the entry point itself never
// does (under lazy module loading the first use of the symbol would).
int noalloc_prepare(vp_ctx* ctx) {
    unsigned char* p = nullptr;
    return scratch_address(ctx, &p);
}

extern "C" int vp_potential_eval_noalloc(vp_ctx* ctx, const vp_nf* nf, const double* f_dev, int32_t d, double* u_dev,
                                         int32_t precision, void* stream) {
    if (!ctx || ctx->magic != 0x56504358) return VP_ERR_STATE;
    if (!nf || nf->magic != 0x56504e46 || nf->ctx != ctx)
        return vp_set_error(ctx, VP_ERR_STATE, "vp_potential_eval_noalloc: bad near-field handle");
    if (!f_dev || !u_dev || d < 1 || d > 256 || (precision != VP_FP64 && precision != VP_MIXED))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_potential_eval_noalloc: bad arguments");
    CurrentDevice guard(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const vp_mesh* mesh = nf->mesh;
    const int64_t N = mesh->N, M = nf->M;
    const int splits = eval_splits(ctx, M, N, 128);   // the split vp_potential_eval uses
    const int dmax = d >= 8 ? 8 : (d >= 4 ? 4 : (d >= 2 ? 2 : 1));   // largest density chunk of the far sum
    const size_t partial_bytes = splits > 1 ? (size_t)splits * d * M * sizeof(double) : 0;
    const size_t off_q = (partial_bytes + 255) & ~(size_t)255;
    const size_t q_bytes = precision == VP_MIXED ? (size_t)N * 2 * dmax * sizeof(float) : 0;
    if (off_q + q_bytes > kScratchBytes)
        return vp_set_error(ctx, VP_ERR_INVALID_ARG,
                            "vp_potential_eval_noalloc: needs " + std::to_string(off_q + q_bytes) +
                                " bytes of scratch, more than the fixed " + std::to_string(kScratchBytes) +
                                " bytes; use vp_potential_eval");
    unsigned char* scratch = nullptr;
    int rc = scratch_address(ctx, &scratch);
    if (rc) return rc;
    // Nothing in the scratch needs to start at zero: every partial sum and
    // every charge is written by this call before it is read.
    double* partial = splits > 1 ? (double*)scratch : u_dev;
    float* qbuf = (float*)(scratch + off_q);
    if (precision == VP_FP64)
        launch_far_fp64(mesh->d_y, mesh->d_W, N, f_dev, d, nf->d_txy, nf->d_tnode, M, partial, splits, s);
    else
        launch_far_ff(nf->src_ff, mesh->d_W, N, f_dev, d, nf->tgt_ff, nf->d_tnode, M, partial, qbuf, splits, s);
    VP_LAUNCH_CHECK(ctx);
    if (splits > 1) launch_reduce_splits(partial, splits, (int64_t)d * M, u_dev, s);
    launch_apply_fp64(nf->d_row, nf->d_ptri, nf->d_C, mesh->nq, f_dev, N, d, M, u_dev, nullptr, s);
    VP_LAUNCH_CHECK(ctx);
    return VP_OK;
}
