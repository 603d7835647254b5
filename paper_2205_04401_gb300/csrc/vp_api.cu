// C ABI of libvp: handles, validation, and the orchestration of the kernels
// for mesh_upload, nearfield_build and potential_eval.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "vp_internal.h"
#include "vp_tables.h"

namespace {

const char* kStatusNames[] = {"VP_OK",          "VP_ERR_INVALID_ARG", "VP_ERR_DEGENERATE_TRI", "VP_ERR_NONFINITE",
                              "VP_ERR_OOM",     "VP_ERR_CUDA",        "VP_ERR_TIMEOUT",        "VP_ERR_NO_DEVICE",
                              "VP_ERR_STATE"};

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Device allocations released at scope exit unless kept.
struct Scratch {
    std::vector<void*> ptrs;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back((void*)*p);
        return e;
    }
    ~Scratch() {
        if (!ptrs.empty()) cudaStreamSynchronize(s);
        for (void* p : ptrs) cudaFree(p);
    }
};

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

void fill_tables(VpTables& t) {
    std::memset(&t, 0, sizeof(t));
    const double* fx[2] = {VP_FAR16_X, VP_FAR19_X};
    const double* fy[2] = {VP_FAR16_Y, VP_FAR19_Y};
    const double* fw[2] = {VP_FAR16_W, VP_FAR19_W};
    const double* fq[2] = {VP_FAR16_Q, VP_FAR19_Q};
    const double* fqm[2] = {VP_FAR16_QM, VP_FAR19_QM};
    const int nq[2] = {16, 19};
    t.far_what[0] = VP_FAR16_WHAT;
    t.far_what[1] = VP_FAR19_WHAT;
    t.far_degree[0] = VP_FAR16_DEGREE;
    t.far_degree[1] = VP_FAR19_DEGREE;
    for (int r = 0; r < 2; r++) {
        t.nq[r] = nq[r];
        for (int k = 0; k < nq[r]; k++) {
            t.fx[r][k] = fx[r][k];
            t.fy[r][k] = fy[r][k];
            t.fw[r][k] = fw[r][k];
            double K[VP_NB];
            koornwinder4(fx[r][k], fy[r][k], K);
            for (int a = 0; a < VP_NB; a++) t.Pk[r][k][a] = fw[r][k] * K[a];
            for (int a = 0; a < VP_NB; a++) t.Q[r][k][a] = fq[r][k * VP_NB + a];
        }
    }
    for (int j = 0; j < VP_NNEAR; j++) {
        t.nx[j] = VP_NEAR33_X[j];
        t.ny[j] = VP_NEAR33_Y[j];
        t.nw[j] = VP_NEAR33_W[j];
    }
    auto split = [](double d) {
        const float h = (float)d;
        return make_float2(h, (float)(d - (double)h));
    };
    for (int j = 0; j < VP_NNEAR; j++) {
        const float2 x = split(VP_NEAR33_X[j]), y = split(VP_NEAR33_Y[j]);
        t.nz2[j] = make_float4(x.x, x.y, y.x, y.y);
        const float2 x3 = split(3.0 * VP_NEAR33_X[j]), y3 = split(3.0 * VP_NEAR33_Y[j]);
        t.nz3[j] = make_float4(x3.x, x3.y, y3.x, y3.y);
        t.nw2[j] = split(VP_NEAR33_W[j]);
    }
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < nq[r]; k++)
            for (int a = 0; a < VP_NB; a++) t.Q2[r][k][a] = split(fqm[r][k * VP_NB + a]);
    for (int r = 0; r < 2; r++) root_leaf_map(fqm[r], nq[r], t.B2[r]);
    for (int j = 0; j < VP_NGL; j++) {
        t.lx2[j] = split(VP_GL16_X[j]);
        t.lw2[j] = split(VP_GL16_W[j]);
    }
    for (int j = 0; j < VP_NGGQ; j++) {
        t.gr2[j] = split(VP_GGQ8_R[j]);
        t.glr2[j] = split(std::log(VP_GGQ8_R[j]));
        t.gwl2[j] = split(VP_GGQ8_W[j] * VP_INV_TWO_PI);
    }
    for (int j = 0; j < VP_NRAD; j++) {
        t.rr2[j] = split(VP_RAD5_R[j]);
        t.ra2[j] = split(VP_RAD5_A[j] * VP_INV_TWO_PI);
        t.rb2[j] = split(VP_RAD5_B[j] * VP_INV_TWO_PI);
    }
    t.near_what = VP_NEAR33_WHAT;
    t.near_degree = VP_NEAR33_DEGREE;
    for (int j = 0; j < VP_NGGQ; j++) {
        t.gr[j] = VP_GGQ8_R[j];
        t.gw[j] = VP_GGQ8_W[j];
        t.glogr[j] = std::log(VP_GGQ8_R[j]);
    }
    for (int j = 0; j < VP_NGL; j++) {
        t.lx[j] = VP_GL16_X[j];
        t.lw[j] = VP_GL16_W[j];
    }
    for (int j = 0; j < 128; j++) {
        t.log_rc[j] = VP_LOG128_RC[j];
        t.log_lc[j] = VP_LOG128_L[j];
    }
    t.ln2 = VP_LN2;
}

bool ctx_ok(const vp_ctx* c) { return c && c->magic == 0x56504358; }
bool mesh_ok(const vp_mesh* m) { return m && m->magic == 0x56504d48; }
bool nf_ok(const vp_nf* n) { return n && n->magic == 0x56504e46; }

int check_flag(vp_ctx* ctx, int32_t* d_flag, cudaStream_t s) {
    int32_t h = 0;
    VP_CUDA_TRY(ctx, cudaMemcpyAsync(&h, d_flag, sizeof(h), cudaMemcpyDeviceToHost, s));
    VP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (h & VP_DEV_ERR_BADIDX) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "triangle vertex index out of range");
    if (h & VP_DEV_ERR_NONFINITE) return vp_set_error(ctx, VP_ERR_NONFINITE, "non-finite coordinate");
    if (h & VP_DEV_ERR_DEGEN) return vp_set_error(ctx, VP_ERR_DEGENERATE_TRI, "triangle with zero area");
    if (h & VP_DEV_ERR_STACK) return vp_set_error(ctx, VP_ERR_CUDA, "near-field subdivision stack overflow");
    if (h & VP_DEV_ERR_CELL) return vp_set_error(ctx, VP_ERR_CUDA, "grid cell list exceeds sort capacity");
    if (h & VP_DEV_ERR_TIMEOUT) return vp_set_error(ctx, VP_ERR_TIMEOUT, "a pipelined kernel timed out waiting for its copies");
    if (h & VP_DEV_ERR_CURVED_CW) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "a curved element is clockwise");
    if (h & VP_DEV_ERR_ALLOC) return vp_set_error(ctx, VP_ERR_OOM, "device allocation failed in the near-field build");
    return VP_OK;
}

int ensure_ws(vp_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return VP_OK;
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    VP_CUDA_TRY(ctx, cudaMalloc(&ctx->ws, want));
    ctx->ws_bytes = want;
    return VP_OK;
}

void free_nf_device(vp_nf* nf) {
    void* ps[] = {nf->d_txy, nf->d_tself, nf->d_tnode, nf->d_row, nf->d_ptri, nf->d_ptgt, nf->d_pkind, nf->d_C, nf->d_C2,
                  nf->src_ff.hi, nf->src_ff.lo, nf->tgt_ff.hi, nf->tgt_ff.lo};
    for (void* p : ps)
        if (p) cudaFree(p);
    tc_plan_free(nf->tc);
    nf->tc = nullptr;
    far_sym_plan_free(nf->sym);
    nf->sym = nullptr;
    fmm_plan_free(nf->fmm);
    nf->fmm = nullptr;
}

}  // namespace

int vp_set_error(vp_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

static const char* kStageNames[ST_COUNT] = {
    "mesh_nodes", "tri_geom", "tri_cells", "cell_sort", "target_cells", "locate", "list_count", "list_fill",
    "weights_self", "weights_near", "ff_split", "far_fp64", "far_ff", "reduce_splits", "apply", "apply_tc",
    "weights_curved", "far_fmm"};

static cudaEvent_t prof_event(vp_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(vp_ctx* ctx, int stage, cudaStream_t s, ProfRec& r) {
    r.stage = -1;
    if (!ctx->prof) return;
    r.stage = stage;
    r.a = prof_event(ctx);
    r.b = prof_event(ctx);
    cudaEventRecord(r.a, s);
}

void prof_end(vp_ctx* ctx, cudaStream_t s, ProfRec& r) {
    if (r.stage < 0) return;
    cudaEventRecord(r.b, s);
    ctx->prof_pending.push_back(r);
}

void prof_collect(vp_ctx* ctx) {
    for (ProfRec& r : ctx->prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->prof_ms[r.stage] += ms;
            ctx->prof_n[r.stage] += 1;
        }
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
}

extern "C" {

const char* vp_status_str(int status) {
    if (status > 0 || status < -8) return "VP_UNKNOWN";
    return kStatusNames[-status];
}

int vp_last_error(const vp_ctx* ctx, char* buf, int32_t len) {
    if (!buf || len <= 0) return VP_ERR_INVALID_ARG;
    const char* m = ctx_ok(ctx) ? ctx->last_error.c_str() : "invalid context";
    std::strncpy(buf, m, (size_t)len - 1);
    buf[len - 1] = 0;
    return VP_OK;
}

int vp_create(vp_ctx** out, int device) {
    if (!out) return VP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return VP_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return VP_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return VP_ERR_NO_DEVICE;
    DevGuard g(device);
    vp_ctx* ctx = new (std::nothrow) vp_ctx();
    if (!ctx) return VP_ERR_OOM;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    fill_tables(ctx->h_tables);
    if (cudaMalloc(&ctx->d_tables, sizeof(VpTables)) != cudaSuccess ||
        cudaMemcpy(ctx->d_tables, &ctx->h_tables, sizeof(VpTables), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&ctx->d_flag, sizeof(int32_t)) != cudaSuccess) {
        vp_destroy(ctx);
        return VP_ERR_OOM;
    }
    // log tables of the float-float units and the no-alloc scratch address:
    // done here so that evaluations never block on a table copy or a module load
    cudaError_t (*const prep[])() = {eval_module_prepare, far_sym_module_prepare, batch_module_prepare,
                                     fmm_module_prepare, weights_module_prepare};
    for (auto fn : prep) {
        const cudaError_t e = fn();
        if (e != cudaSuccess) {
            vp_destroy(ctx);
            return e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA;
        }
    }
    if (int rc = noalloc_prepare(ctx)) {
        vp_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return VP_OK;
}

int vp_set_far_sym_cap(vp_ctx* ctx, int64_t bytes) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (bytes < ((int64_t)1 << 20) || bytes > ((int64_t)1 << 40))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_set_far_sym_cap: bytes outside [1 MiB, 1 TiB]");
    ctx->far_sym_cap_bytes = bytes;
    return VP_OK;
}

int vp_ctx_memory(const vp_ctx* ctx, int64_t* workspace_bytes, int64_t* staging_bytes) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (workspace_bytes) *workspace_bytes = (int64_t)ctx->ws_bytes;
    if (staging_bytes) *staging_bytes = (int64_t)ctx->stage_bytes;
    return VP_OK;
}

void vp_destroy(vp_ctx* ctx) {
    if (!ctx_ok(ctx)) return;
    DevGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->d_tables) cudaFree(ctx->d_tables);
    far_rules_free(ctx);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->stage) cudaFree(ctx->stage);
    prof_collect(ctx);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    ctx->magic = 0;
    delete ctx;
}

// -------------------------------------------------------------------- mesh
// Curves of vp_mesh_upload_curved, already on the device and owned by the
// new mesh from the call on (released with it, or on failure).
struct CurvesIn {
    int32_t* d_cidx = nullptr;
    double* d_coef = nullptr;
    double* d_dcoef = nullptr;
    int64_t ncurve = 0;
    int K = 0;
};

static int mesh_upload_impl(vp_ctx* ctx, const double* d_vxy, int64_t nv, const int32_t* d_tri, int64_t nt,
                            int32_t rule, cudaStream_t s, vp_mesh** out, CurvesIn cin = CurvesIn()) {
    vp_mesh* m = new (std::nothrow) vp_mesh();
    if (!m) {
        if (cin.d_cidx) cudaFree(cin.d_cidx);
        if (cin.d_coef) cudaFree(cin.d_coef);
        if (cin.d_dcoef) cudaFree(cin.d_dcoef);
        return VP_ERR_OOM;
    }
    m->ctx = ctx;
    m->d_cidx = cin.d_cidx;
    m->d_coef = cin.d_coef;
    m->d_dcoef = cin.d_dcoef;
    m->ncurve = cin.ncurve;
    m->K = cin.K;
    m->nt = nt;
    m->nv = nv;
    int rc = far_rule_get(ctx, rule, &m->rule);
    if (rc != VP_OK) {
        vp_mesh_release(m);
        return rc;
    }
    m->nq = m->rule.dev.nq;
    m->N = nt * m->nq;
    double* d_red = nullptr;
    cudaError_t e = dev_alloc(&m->d_tv, 6 * nt);
    if (e == cudaSuccess) e = dev_alloc(&m->d_J, nt);
    if (e == cudaSuccess) e = dev_alloc(&m->d_y, 2 * m->N);
    if (e == cudaSuccess) e = dev_alloc(&m->d_W, m->N);
    if (e == cudaSuccess) e = dev_alloc(&d_red, 8);
    if (e != cudaSuccess) rc = vp_set_error(ctx, VP_ERR_OOM, "vp_mesh_upload: device allocation failed");
    if (rc == VP_OK) {
        cudaMemsetAsync(ctx->d_flag, 0, sizeof(int32_t), s);
        PROF(ctx, ST_MESH_NODES, s,
             launch_mesh_nodes(d_vxy, nv, d_tri, nt, m->rule.dev, m->d_tv, m->d_J, m->d_y, m->d_W, ctx->d_flag, s));
        if (m->d_cidx)
            PROF(ctx, ST_MESH_NODES, s,
                 launch_mesh_nodes_curved(d_vxy, nv, d_tri, nt, mesh_curves(m), m->rule.dev, m->d_tv, m->d_y, m->d_W,
                                          ctx->d_flag, s));
        launch_bbox_reduce(d_vxy, nv, 2, d_red, s);
        if (m->d_cidx) launch_bbox_reduce(m->d_y, m->N, 2, d_red + 4, s);   // nodes on the curved sides' bulges
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) rc = vp_set_error(ctx, VP_ERR_CUDA, cudaGetErrorString(le));
        else rc = check_flag(ctx, ctx->d_flag, s);
        double hb[8];
        if (rc == VP_OK && cudaMemcpy(hb, d_red, 8 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = vp_set_error(ctx, VP_ERR_CUDA, "vp_mesh_upload: bbox copy failed");
        if (rc == VP_OK) {
            for (int i = 0; i < 4; i++) m->bbox[i] = hb[i];
            if (m->d_cidx) {
                m->bbox[0] = std::min(m->bbox[0], hb[4]);
                m->bbox[1] = std::min(m->bbox[1], hb[5]);
                m->bbox[2] = std::max(m->bbox[2], hb[6]);
                m->bbox[3] = std::max(m->bbox[3], hb[7]);
            }
        }
    }
    if (d_red) cudaFree(d_red);
    if (rc != VP_OK) {
        vp_mesh_release(m);
        return rc;
    }
    *out = m;
    return VP_OK;
}

int vp_mesh_upload(vp_ctx* ctx, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, int32_t rule,
                   void* stream, vp_mesh** out) {
    if (out) *out = nullptr;
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!out || !vxy || !tri || nv < 3 || nt < 1 || !far_rule_valid(rule))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload: bad arguments");
    if (nt > (int64_t)INT32_MAX / far_rule_nq(rule))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload: too many triangles");
    for (int64_t i = 0; i < 2 * nv; i++)
        if (!std::isfinite(vxy[i])) return vp_set_error(ctx, VP_ERR_NONFINITE, "vp_mesh_upload: non-finite vertex");
    for (int64_t i = 0; i < 3 * nt; i++)
        if (tri[i] < 0 || tri[i] >= nv) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload: index out of range");
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    double* d_vxy;
    int32_t* d_tri;
    if (sc.alloc(&d_vxy, 2 * nv) != cudaSuccess || sc.alloc(&d_tri, 3 * nt) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_OOM, "vp_mesh_upload: device allocation failed");
    VP_CUDA_TRY(ctx, cudaMemcpyAsync(d_vxy, vxy, 2 * nv * sizeof(double), cudaMemcpyHostToDevice, s));
    VP_CUDA_TRY(ctx, cudaMemcpyAsync(d_tri, tri, 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    return mesh_upload_impl(ctx, d_vxy, nv, d_tri, nt, rule, s, out);
}

int vp_mesh_upload_dev(vp_ctx* ctx, const double* vxy_dev, int64_t nv, const int32_t* tri_dev, int64_t nt,
                       int32_t rule, void* stream, vp_mesh** out) {
    if (out) *out = nullptr;
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!out || !vxy_dev || !tri_dev || nv < 3 || nt < 1 || !far_rule_valid(rule))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload_dev: bad arguments");
    if (nt > (int64_t)INT32_MAX / far_rule_nq(rule))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload_dev: too many triangles");
    DevGuard g(ctx->device);
    return mesh_upload_impl(ctx, vxy_dev, nv, tri_dev, nt, rule, (cudaStream_t)stream, out);
}

int vp_mesh_upload_curved(vp_ctx* ctx, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt,
                          const int32_t* cidx, const double* coef, int64_t ncurve, int32_t K, int32_t rule,
                          void* stream, vp_mesh** out) {
    if (out) *out = nullptr;
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!out || !vxy || !tri || !cidx || nv < 3 || nt < 1 || ncurve < 0 || (ncurve > 0 && !coef) || K < 0 ||
        K > VP_MAX_CHEB || !far_rule_valid(rule))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload_curved: bad arguments");
    if (nt > (int64_t)INT32_MAX / far_rule_nq(rule)) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload_curved: too many triangles");
    for (int64_t i = 0; i < 2 * nv; i++)
        if (!std::isfinite(vxy[i])) return vp_set_error(ctx, VP_ERR_NONFINITE, "vp_mesh_upload_curved: non-finite vertex");
    for (int64_t i = 0; i < 3 * nt; i++)
        if (tri[i] < 0 || tri[i] >= nv)
            return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload_curved: index out of range");
    for (int64_t i = 0; i < nt; i++)
        if (cidx[i] < -1 || cidx[i] >= ncurve)
            return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_mesh_upload_curved: curve index out of range");
    const int64_t ncoef = ncurve * 2 * (K + 1);
    for (int64_t i = 0; i < ncoef; i++)
        if (!std::isfinite(coef[i]))
            return vp_set_error(ctx, VP_ERR_NONFINITE, "vp_mesh_upload_curved: non-finite curve coefficient");
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    double* d_vxy;
    int32_t* d_tri;
    if (sc.alloc(&d_vxy, 2 * nv) != cudaSuccess || sc.alloc(&d_tri, 3 * nt) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_OOM, "vp_mesh_upload_curved: device allocation failed");
    CurvesIn cin;
    cin.ncurve = ncurve;
    cin.K = K;
    // Chebyshev coefficients of dD/dt (t = 2 xi - 1), per curve and coordinate:
    // c_{K-1} = 2 K a_K, c_{k-1} = c_{k+1} + 2 k a_k, then c_0 / 2
    std::vector<double> dcoef((size_t)ncoef, 0.0);
    for (int64_t c = 0; c < 2 * ncurve; c++) {
        const double* a = coef + c * (K + 1);
        double* d = dcoef.data() + c * (K + 1);
        for (int k = K; k >= 1; k--) d[k - 1] = (k + 1 <= K ? d[k + 1] : 0.0) + 2.0 * k * a[k];
        d[0] *= 0.5;
    }
    if (dev_alloc(&cin.d_cidx, nt) != cudaSuccess ||
        (ncoef > 0 && (dev_alloc(&cin.d_coef, ncoef) != cudaSuccess || dev_alloc(&cin.d_dcoef, ncoef) != cudaSuccess))) {
        if (cin.d_cidx) cudaFree(cin.d_cidx);
        if (cin.d_coef) cudaFree(cin.d_coef);
        return vp_set_error(ctx, VP_ERR_OOM, "vp_mesh_upload_curved: device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(d_vxy, vxy, 2 * nv * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tri, tri, 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cin.d_cidx, cidx, nt * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && ncoef > 0)
        e = cudaMemcpyAsync(cin.d_coef, coef, ncoef * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && ncoef > 0)
        e = cudaMemcpyAsync(cin.d_dcoef, dcoef.data(), ncoef * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host arrays are read during the call only
    if (e != cudaSuccess) {
        cudaFree(cin.d_cidx);
        if (cin.d_coef) cudaFree(cin.d_coef);
        if (cin.d_dcoef) cudaFree(cin.d_dcoef);
        return vp_set_error(ctx, VP_ERR_CUDA, std::string("vp_mesh_upload_curved: copy failed: ") + cudaGetErrorString(e));
    }
    return mesh_upload_impl(ctx, d_vxy, nv, d_tri, nt, rule, s, out, cin);
}

int vp_mesh_info(const vp_mesh* mesh, int64_t* n_tri, int64_t* n_nodes, int32_t* nq) {
    if (!mesh_ok(mesh)) return VP_ERR_STATE;
    if (n_tri) *n_tri = mesh->nt;
    if (n_nodes) *n_nodes = mesh->N;
    if (nq) *nq = mesh->nq;
    return VP_OK;
}

int vp_mesh_nodes(const vp_mesh* mesh, double* yxy_dev, double* w_dev, void* stream) {
    if (!mesh_ok(mesh)) return VP_ERR_STATE;
    DevGuard g(mesh->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (yxy_dev) VP_CUDA_TRY(mesh->ctx, cudaMemcpyAsync(yxy_dev, mesh->d_y, 2 * mesh->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (w_dev) VP_CUDA_TRY(mesh->ctx, cudaMemcpyAsync(w_dev, mesh->d_W, mesh->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return VP_OK;
}

void vp_mesh_release(vp_mesh* mesh) {
    if (!mesh_ok(mesh)) return;
    DevGuard g(mesh->ctx->device);
    cudaDeviceSynchronize();
    void* ps[] = {mesh->d_tv, mesh->d_J, mesh->d_y, mesh->d_W, mesh->d_cidx, mesh->d_coef, mesh->d_dcoef};
    for (void* p : ps)
        if (p) cudaFree(p);
    mesh->magic = 0;
    delete mesh;
}

// -------------------------------------------------------------- near field
int vp_nf_params_default(vp_nf_params* out) {
    if (!out) return VP_ERR_INVALID_ARG;
    out->eps = 1e-12;
    out->c_far = 1.0;
    out->c_near = 12.0;   // Table "C_N values": C_12 = 12 for the order-12 near rule
    out->depth_cap = 30;
    out->flags = 0;
    return VP_OK;
}

int vp_nearfield_build(vp_ctx* ctx, const vp_mesh* mesh, int32_t node_targets, const double* txy_dev, int64_t m,
                       const vp_nf_params* params, void* stream, vp_nf** out) {
    if (out) *out = nullptr;
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!mesh_ok(mesh) || mesh->ctx != ctx) return vp_set_error(ctx, VP_ERR_STATE, "vp_nearfield_build: bad mesh");
    if (!out || m < 0 || (m > 0 && !txy_dev)) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_nearfield_build: bad arguments");
    const int64_t N = mesh->N, nt = mesh->nt;
    const int nq = mesh->nq;
    const int64_t M = (node_targets ? N : 0) + m;
    if (M < 1 || M > (int64_t)INT32_MAX) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_nearfield_build: no targets");
    vp_nf_params prm;
    vp_nf_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.eps >= 1e-15 && prm.eps <= 1e-2) || !(prm.c_far > 0) || !(prm.c_near > 0) || prm.depth_cap < 0 ||
        prm.depth_cap > 30 || (prm.flags & ~VP_NF_FP64_WEIGHTS))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_nearfield_build: bad params");
    auto t_start = std::chrono::steady_clock::now();
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    vp_nf* nf = new (std::nothrow) vp_nf();
    if (!nf) return VP_ERR_OOM;
    nf->ctx = ctx;
    nf->mesh = mesh;
    nf->M = M;
    nf->n_extra = m;
    nf->node_targets = node_targets ? 1 : 0;
    nf->params = prm;
    int rc = VP_OK;
#define NF_FAIL(code, msg)                          \
    do {                                            \
        rc = vp_set_error(ctx, (code), (msg));      \
        goto fail;                                  \
    } while (0)
#define NF_CUDA(expr)                                                                           \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess)                                                                  \
            NF_FAIL(_e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA,                 \
                    std::string(#expr) + ": " + cudaGetErrorString(_e));                        \
    } while (0)
    {
        Scratch sc(s);
        double *d_R, *d_bbox, *d_red;
        double h_red[4], h_tb[4];
        GridDev gd;
        int64_t ncell, nentries = 0;
        int32_t *d_cnt, *d_cell_tri, *d_tcell, *d_tcnt, *d_order, *d_count, *d_near_idx, *d_self_idx, *d_pstat, *d_pcap;
        int32_t *d_max;
        int64_t *d_cell_start, *d_cursor, *d_tstart;
        unsigned long long* d_u64;
        unsigned long long h_u64[4] = {0, 0, 0, 0};
        int32_t *d_cnear_idx = nullptr, *d_cself_idx = nullptr;
        uint32_t* d_lcache = nullptr;
        constexpr int LIST_CAP = 48;
        char* d_f2ws;
        int32_t h_max = 0;
        std::vector<double> hb;
        std::vector<double> sizes;
        double W_, H_, hc;
        int64_t nx, ny;
        WeightsArgs wa;
        int64_t n_near, n_self;

        NF_CUDA(dev_alloc(&nf->d_txy, 2 * M));
        NF_CUDA(dev_alloc(&nf->d_tnode, M));
        NF_CUDA(dev_alloc(&nf->d_tself, M));
        launch_targets_init(mesh->d_y, N, nq, nf->node_targets, txy_dev, m, nf->d_txy, nf->d_tnode, nf->d_tself, s);
        NF_CUDA(cudaGetLastError());

        // per-triangle ellipse parameter and bounding boxes
        NF_CUDA(sc.alloc(&d_R, nt));
        NF_CUDA(sc.alloc(&d_bbox, 4 * nt));
        NF_CUDA(sc.alloc(&d_red, 8));
        PROF(ctx, ST_TRI_GEOM, s,
             launch_tri_geom(mesh->d_tv, mesh->d_J, nt, mesh->rule.what, mesh->rule.degree, prm.eps, prm.c_far, d_R,
                             d_bbox, s));
        if (mesh->d_cidx) launch_curved_bbox(nt, mesh_curves(mesh), d_bbox, s);
        launch_bbox_reduce(d_bbox, nt, 4, d_red, s);
        launch_bbox_reduce(nf->d_txy, M, 2, d_red + 4, s);
        NF_CUDA(cudaGetLastError());
        hb.resize(4 * nt);
        NF_CUDA(cudaMemcpyAsync(hb.data(), d_bbox, 4 * nt * sizeof(double), cudaMemcpyDeviceToHost, s));
        NF_CUDA(cudaMemcpyAsync(h_red, d_red, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        NF_CUDA(cudaMemcpyAsync(h_tb, d_red + 4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        NF_CUDA(cudaStreamSynchronize(s));
        if (!std::isfinite(h_tb[0]) || !std::isfinite(h_tb[1]) || !std::isfinite(h_tb[2]) || !std::isfinite(h_tb[3]))
            NF_FAIL(VP_ERR_NONFINITE, "vp_nearfield_build: non-finite target");

        // grid: cell = half the 25th percentile of the triangles' box sizes
        sizes.resize(nt);
        for (int64_t t = 0; t < nt; t++) sizes[t] = std::max(hb[4 * t + 2] - hb[4 * t], hb[4 * t + 3] - hb[4 * t + 1]);
        std::nth_element(sizes.begin(), sizes.begin() + nt / 4, sizes.end());
        W_ = h_red[2] - h_red[0];
        H_ = h_red[3] - h_red[1];
        hc = std::max(0.5 * sizes[nt / 4], 1e-300);
        hc = std::max(hc, std::max(W_, H_) / 4096.0);
        nx = std::max<int64_t>(1, (int64_t)std::ceil(W_ / hc));
        ny = std::max<int64_t>(1, (int64_t)std::ceil(H_ / hc));
        while (nx * ny > ((int64_t)1 << 24)) {
            hc *= 1.5;
            nx = std::max<int64_t>(1, (int64_t)std::ceil(W_ / hc));
            ny = std::max<int64_t>(1, (int64_t)std::ceil(H_ / hc));
        }
        ncell = nx * ny;
        gd.ox = h_red[0];
        gd.oy = h_red[1];
        gd.h = hc;
        gd.nx = (int32_t)nx;
        gd.ny = (int32_t)ny;
        gd.cell_start = nullptr;
        gd.cell_tri = nullptr;

        // triangles -> cells (sorted per cell)
        NF_CUDA(sc.alloc(&d_cnt, ncell));
        NF_CUDA(sc.alloc(&d_cell_start, ncell + 1));
        NF_CUDA(sc.alloc(&d_cursor, ncell + 1));
        NF_CUDA(sc.alloc(&d_max, 1));
        NF_CUDA(cudaMemsetAsync(d_cnt, 0, ncell * sizeof(int32_t), s));
        PROF(ctx, ST_TRI_CELLS, s, launch_tri_cell_count(d_bbox, nt, gd, d_cnt, s));
        rc = vp_exclusive_scan_i32(ctx, d_cnt, d_cell_start, ncell, s);
        if (rc) goto fail;
        launch_max_i32(d_cnt, ncell, d_max, s);
        NF_CUDA(cudaMemcpyAsync(&nentries, d_cell_start + ncell, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        NF_CUDA(cudaMemcpyAsync(&h_max, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        NF_CUDA(cudaStreamSynchronize(s));
        if (h_max > 16384) NF_FAIL(VP_ERR_CUDA, "vp_nearfield_build: a grid cell holds more than 16384 triangles");
        NF_CUDA(sc.alloc(&d_cell_tri, nentries));
        NF_CUDA(cudaMemcpyAsync(d_cursor, d_cell_start, (ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        PROF(ctx, ST_TRI_CELLS, s, launch_tri_cell_fill(d_bbox, nt, gd, d_cursor, d_cell_tri, s));
        gd.cell_start = d_cell_start;
        gd.cell_tri = d_cell_tri;
        NF_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int32_t), s));
        PROF(ctx, ST_CELL_SORT, s, launch_cell_sort(gd, ncell, h_max, d_cell_tri, ctx->d_flag, s));
        NF_CUDA(cudaGetLastError());

        // targets -> cells, processing order grouped by cell
        NF_CUDA(sc.alloc(&d_tcell, M));
        NF_CUDA(sc.alloc(&d_tcnt, ncell));
        NF_CUDA(sc.alloc(&d_tstart, ncell + 1));
        NF_CUDA(sc.alloc(&d_order, M));
        NF_CUDA(cudaMemsetAsync(d_tcnt, 0, ncell * sizeof(int32_t), s));
        PROF(ctx, ST_TARGET_CELLS, s, launch_target_cells(nf->d_txy, M, gd, d_tcell, d_tcnt, s));
        rc = vp_exclusive_scan_i32(ctx, d_tcnt, d_tstart, ncell, s);
        if (rc) goto fail;
        PROF(ctx, ST_TARGET_CELLS, s, launch_target_order(d_tcell, M, d_tstart, d_order, s));

        // S(x) for extra targets, then the two list passes
        if (mesh->d_cidx)
            PROF(ctx, ST_LOCATE, s,
                 launch_locate_curved(mesh->d_tv, mesh_curves(mesh), nf->d_txy, d_order, d_tcell, M, gd, nf->d_tself, s));
        else
            PROF(ctx, ST_LOCATE, s, launch_locate(mesh->d_tv, nf->d_txy, d_order, d_tcell, M, gd, nf->d_tself, s));
        NF_CUDA(sc.alloc(&d_count, M));
        // the counting pass keeps up to LIST_CAP entries per target for the filling pass
        if (sc.alloc(&d_lcache, (size_t)M * LIST_CAP) != cudaSuccess) {
            cudaGetLastError();
            d_lcache = nullptr;
        }
        PROF(ctx, ST_LIST_COUNT, s,
             launch_list_pass(mesh->d_tv, d_R, mesh->rule.degree, nf->d_txy, nf->d_tself, d_order, d_tcell, M, gd,
                              d_count, nullptr, nullptr, nullptr, nullptr, d_lcache, LIST_CAP, s));
        NF_CUDA(dev_alloc(&nf->d_row, M + 1));
        rc = vp_exclusive_scan_i32(ctx, d_count, nf->d_row, M, s);
        if (rc) goto fail;
        NF_CUDA(cudaMemcpyAsync(&nf->P, nf->d_row + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        NF_CUDA(cudaStreamSynchronize(s));
        if (nf->P > (int64_t)INT32_MAX) NF_FAIL(VP_ERR_INVALID_ARG, "vp_nearfield_build: more than 2^31 pairs");
        // pair arrays carry 16 bytes of padding (the streamed apply copies
        // whole 16-byte units)
        NF_CUDA(dev_alloc(&nf->d_ptri, nf->P + 4));
        NF_CUDA(dev_alloc(&nf->d_ptgt, nf->P + 4));
        NF_CUDA(dev_alloc(&nf->d_pkind, nf->P));
        NF_CUDA(dev_alloc(&nf->d_C, nf->P * nq));
        PROF(ctx, ST_LIST_FILL, s,
             launch_list_pass(mesh->d_tv, d_R, mesh->rule.degree, nf->d_txy, nf->d_tself, d_order, d_tcell, M, gd,
                              nullptr, nf->d_row, nf->d_ptri, nf->d_ptgt, nf->d_pkind, d_lcache, LIST_CAP, s));
        NF_CUDA(cudaGetLastError());

        // correction weights
        NF_CUDA(sc.alloc(&d_near_idx, nf->P));
        NF_CUDA(sc.alloc(&d_self_idx, nf->P));
        NF_CUDA(sc.alloc(&d_u64, 4));
        NF_CUDA(sc.alloc(&d_pstat, nf->P));
        NF_CUDA(sc.alloc(&d_pcap, nf->P));
        if (mesh->d_cidx) {
            // pairs on curved triangles get their own lists and kernels
            NF_CUDA(sc.alloc(&d_cnear_idx, nf->P));
            NF_CUDA(sc.alloc(&d_cself_idx, nf->P));
            launch_split_pairs4(nf->d_pkind, nf->d_ptri, mesh_curves(mesh), nf->P, d_near_idx, d_self_idx, d_cnear_idx,
                                d_cself_idx, d_u64, s);
            NF_CUDA(cudaMemcpyAsync(h_u64, d_u64, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        } else {
            launch_split_pairs(nf->d_pkind, nf->P, d_near_idx, d_self_idx, d_u64, s);
            NF_CUDA(cudaMemcpyAsync(h_u64, d_u64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        }
        NF_CUDA(cudaStreamSynchronize(s));
        n_near = (int64_t)h_u64[0];
        n_self = (int64_t)h_u64[1];
        wa.tab = ctx->d_tables;
        wa.Q = mesh->rule.dev.Q;
        wa.Q2 = mesh->rule.dev.Q2;
        wa.B2 = mesh->rule.dev.B2;
        wa.nq = nq;
        wa.tv = mesh->d_tv;
        wa.J = mesh->d_J;
        wa.y = mesh->d_y;
        wa.W = mesh->d_W;
        wa.txy = nf->d_txy;
        wa.tnode = nf->d_tnode;
        wa.ptri = nf->d_ptri;
        wa.ptgt = nf->d_ptgt;
        wa.C = nf->d_C;
        wa.pstat = d_pstat;
        wa.pcap = d_pcap;
        wa.flag = ctx->d_flag;
        wa.eps = prm.eps;
        wa.c_near = prm.c_near;
        wa.depth_cap = prm.depth_cap;
        wa.fp64 = (prm.flags & VP_NF_FP64_WEIGHTS) ? 1 : 0;
        if (!wa.fp64) NF_CUDA(dev_alloc(&nf->d_C2, nf->P * nq + 2));
        wa.C2 = nf->d_C2;
        wa.nt = nt;
        wa.M = M;
        wa.N = N;
        NF_CUDA(sc.alloc(&d_f2ws, (int64_t)weights_f2_bytes(nt, M, N, n_near)));
        wa.f2_ws = d_f2ws;
        launch_weights(wa, d_self_idx, n_self, d_near_idx, n_near, s, ctx);
        if (mesh->d_cidx)
            launch_weights_curved(wa, mesh_curves(mesh), d_cself_idx, (int64_t)h_u64[3], d_cnear_idx,
                                  (int64_t)h_u64[2], s, ctx);
        NF_CUDA(cudaGetLastError());

        // statistics
        nf->stats.n_targets = M;
        nf->stats.n_nodes = N;
        nf->stats.n_pairs = nf->P;
        nf->stats.n_near = n_near + (int64_t)h_u64[2];
        nf->stats.n_self = n_self + (int64_t)h_u64[3];
        nf->stats.outside = M - nf->stats.n_self;
        {
            // leaves (near pairs) and panels (self pairs), depth-capped leaves
            unsigned long long h3[3];
            launch_sum_by_kind(d_pstat, nf->d_pkind, d_pcap, nf->P, d_u64, s);
            NF_CUDA(cudaMemcpyAsync(h3, d_u64, sizeof(h3), cudaMemcpyDeviceToHost, s));
            NF_CUDA(cudaStreamSynchronize(s));
            nf->stats.near_leaves = (int64_t)h3[0];
            nf->stats.self_panels = (int64_t)h3[1];
            nf->stats.depth_capped = (int64_t)h3[2];
        }

        // float-float coordinates for the mixed far sum: origin at the centre
        // of the node/target box, hi parts on the grid q = 2^(e - 22) with
        // 2^e > the largest offset: |hi| / q <= 2^22 and every hi difference
        // is a multiple of q below 2^24 q, hence exact in FP32.
        {
            const double ox = 0.5 * (std::min(mesh->bbox[0], h_tb[0]) + std::max(mesh->bbox[2], h_tb[2]));
            const double oy = 0.5 * (std::min(mesh->bbox[1], h_tb[1]) + std::max(mesh->bbox[3], h_tb[3]));
            double ext = 0;
            ext = std::max(ext, std::fabs(mesh->bbox[0] - ox));
            ext = std::max(ext, std::fabs(mesh->bbox[2] - ox));
            ext = std::max(ext, std::fabs(mesh->bbox[1] - oy));
            ext = std::max(ext, std::fabs(mesh->bbox[3] - oy));
            ext = std::max(ext, std::fabs(h_tb[0] - ox));
            ext = std::max(ext, std::fabs(h_tb[2] - ox));
            ext = std::max(ext, std::fabs(h_tb[1] - oy));
            ext = std::max(ext, std::fabs(h_tb[3] - oy));
            int e = 0;
            std::frexp(std::max(ext, 1e-300), &e);   // ext < 2^e
            nf->ff_origin[0] = ox;
            nf->ff_origin[1] = oy;
            nf->ff_scale = std::ldexp(1.0, e - 22);
            NF_CUDA(dev_alloc(&nf->src_ff.hi, 2 * N));
            NF_CUDA(dev_alloc(&nf->src_ff.lo, 2 * N));
            NF_CUDA(dev_alloc(&nf->tgt_ff.hi, 2 * M));
            NF_CUDA(dev_alloc(&nf->tgt_ff.lo, 2 * M));
            PROF(ctx, ST_FF_SPLIT, s, launch_ff_split(mesh->d_y, N, ox, oy, nf->ff_scale, nf->src_ff, s);
                 launch_ff_split(nf->d_txy, M, ox, oy, nf->ff_scale, nf->tgt_ff, s));
            NF_CUDA(cudaGetLastError());
        }
        rc = check_flag(ctx, ctx->d_flag, s);
        if (rc) goto fail;
    }
    nf->stats.bytes_device = (int64_t)(M * (16 + 4 + 4 + 8 + 16 + 16) + 8 + nf->P * (4 + 4 + 1 + 8 * nq) + N * 16);
    nf->stats.build_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    *out = nf;
    return VP_OK;
fail:
    cudaStreamSynchronize(s);
    free_nf_device(nf);
    nf->magic = 0;
    delete nf;
    return rc;
#undef NF_FAIL
#undef NF_CUDA
}

int vp_nearfield_build_host(vp_ctx* ctx, const vp_mesh* mesh, int32_t node_targets, const double* txy_host,
                            int64_t m, const vp_nf_params* params, void* stream, vp_nf** out) {
    if (out) *out = nullptr;
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (m < 0 || (m > 0 && !txy_host))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_nearfield_build_host: bad arguments");
    if (m == 0) return vp_nearfield_build(ctx, mesh, node_targets, nullptr, 0, params, stream, out);
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t tb = (size_t)m * 2 * sizeof(double);
    if (tb > ctx->stage_bytes) {
        if (ctx->stage) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
        }
        VP_CUDA_TRY(ctx, cudaMalloc(&ctx->stage, tb));
        ctx->stage_bytes = tb;
    }
    VP_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->stage, txy_host, tb, cudaMemcpyHostToDevice, s));
    // the build copies the targets into its own arrays and synchronises `stream`
    return vp_nearfield_build(ctx, mesh, node_targets, ctx->stage, m, params, stream, out);
}

int vp_nf_stats(const vp_nf* nf, vp_nf_stats_t* out) {
    if (!nf_ok(nf)) return VP_ERR_STATE;
    if (!out) return VP_ERR_INVALID_ARG;
    *out = nf->stats;
    return VP_OK;
}

int vp_nf_lists(const vp_nf* nf, int64_t* row_ptr_dev, int32_t* tri_dev, uint8_t* kind_dev, int32_t* tself_dev,
                void* stream) {
    if (!nf_ok(nf)) return VP_ERR_STATE;
    vp_ctx* ctx = nf->ctx;
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (row_ptr_dev) VP_CUDA_TRY(ctx, cudaMemcpyAsync(row_ptr_dev, nf->d_row, (nf->M + 1) * 8, cudaMemcpyDeviceToDevice, s));
    if (tri_dev && nf->P) VP_CUDA_TRY(ctx, cudaMemcpyAsync(tri_dev, nf->d_ptri, nf->P * 4, cudaMemcpyDeviceToDevice, s));
    if (kind_dev && nf->P) VP_CUDA_TRY(ctx, cudaMemcpyAsync(kind_dev, nf->d_pkind, nf->P, cudaMemcpyDeviceToDevice, s));
    if (tself_dev) VP_CUDA_TRY(ctx, cudaMemcpyAsync(tself_dev, nf->d_tself, nf->M * 4, cudaMemcpyDeviceToDevice, s));
    return VP_OK;
}

int vp_nf_weights(const vp_nf* nf, double* w_dev, void* stream) {
    if (!nf_ok(nf)) return VP_ERR_STATE;
    vp_ctx* ctx = nf->ctx;
    DevGuard g(ctx->device);
    if (w_dev && nf->P)
        VP_CUDA_TRY(ctx, cudaMemcpyAsync(w_dev, nf->d_C, nf->P * nf->mesh->nq * sizeof(double), cudaMemcpyDeviceToDevice,
                                         (cudaStream_t)stream));
    return VP_OK;
}

void vp_nf_release(vp_nf* nf) {
    if (!nf_ok(nf)) return;
    DevGuard g(nf->ctx->device);
    cudaDeviceSynchronize();
    free_nf_device(nf);
    nf->magic = 0;
    delete nf;
}

// ------------------------------------------------------------- evaluation
}  // extern "C"

int eval_splits(const vp_ctx* ctx, int64_t M, int64_t N, int threads) {
    const int64_t blocks = (M + threads - 1) / threads;
    const int64_t want = 4LL * ctx->sm_count;
    int64_t s = (want + blocks - 1) / blocks;
    s = std::min<int64_t>(s, std::max<int64_t>(1, N / 1024));
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 64));
}

// Layout: [split partials][far-sum scratch][apply scratch].  Sized for both
// far-sum paths (the symmetric one runs once its plan exists).
static size_t eval_layout(const vp_ctx* ctx, const vp_nf* nf, int d, int precision, bool sym, size_t* off_q,
                          size_t* off_t) {
    const int64_t N = nf->mesh->N, M = nf->M;
    const bool fmm = precision == VP_MIXED_FMM;
    const int splits = (sym || fmm) ? 1 : eval_splits(ctx, M, N, 128);
    const size_t partial_bytes = splits > 1 ? (size_t)splits * d * M * sizeof(double) : 0;
    *off_q = (partial_bytes + 255) & ~(size_t)255;
    const size_t q_bytes = fmm ? fmm_ws_bytes(nf, d)
                               : sym ? far_sym_ws_bytes(ctx, nf) : (precision != VP_FP64 ? (size_t)N * 16 * sizeof(float) : 0);
    *off_t = (*off_q + q_bytes + 255) & ~(size_t)255;
    const bool mixed_apply = precision == VP_MIXED || precision == VP_MIXED_FMM;
    size_t f2_bytes = mixed_apply && d < APPLY_MANY_MIN_D ? (size_t)N * d * sizeof(float2) : 0;
    if (mixed_apply && d == 1) f2_bytes = std::max(f2_bytes, apply_stream_ws_bytes(N, nf->P));
    return *off_t + std::max(precision == VP_MIXED_TC ? tc_ws_bytes(nf) : apply_ws_bytes(N, d), f2_bytes) + 256;
}

size_t eval_ws_bytes(const vp_ctx* ctx, const vp_nf* nf, int d, int precision) {
    size_t oq, ot;
    size_t b = eval_layout(ctx, nf, d, precision, false, &oq, &ot);
    if ((precision == VP_MIXED || precision == VP_MIXED_TC) && far_sym_applicable(nf, d))
        b = std::max(b, eval_layout(ctx, nf, d, precision, true, &oq, &ot));
    return b;
}

// The evaluation with caller-provided workspace (at least eval_ws_bytes).
int eval_impl(vp_ctx* ctx, const vp_nf* nf, const double* f_dev, int32_t d, double* u_dev, int32_t precision,
              cudaStream_t s, void* ws, bool profile) {
    const vp_mesh* mesh = nf->mesh;
    const int64_t N = mesh->N, M = nf->M;
    const bool fmm = precision == VP_MIXED_FMM;
    const bool sym = (precision == VP_MIXED || precision == VP_MIXED_TC) && far_sym_applicable(nf, d) && nf->sym;
    const int splits = (sym || fmm) ? 1 : eval_splits(ctx, M, N, 128);
    size_t off_q, off_t;
    eval_layout(ctx, nf, d, precision, sym, &off_q, &off_t);
    double* partial = splits > 1 ? (double*)ws : u_dev;
    float* qbuf = (float*)((char*)ws + off_q);
    void* apply_ws = (char*)ws + off_t;
    double* fT = apply_ws_bytes(N, d) ? (double*)apply_ws : nullptr;
    const bool prof_saved = ctx->prof;
    if (!profile) ctx->prof = false;
    // the streamed apply (one density, mixed) gathers the density as
    // float-float pairs: the direct far sum's charge preparation writes them
    const bool stream_apply = precision != VP_MIXED_TC && mesh->rule.builtin >= 0 &&
                              (precision == VP_MIXED || fmm) && d == 1 && nf->d_C2;
    float2* f2out = stream_apply && !fmm ? (float2*)apply_ws : nullptr;
    if (precision == VP_FP64)
        PROF(ctx, ST_FAR_FP64, s,
             launch_far_fp64(mesh->d_y, mesh->d_W, N, f_dev, d, nf->d_txy, nf->d_tnode, M, partial, splits, s));
    else if (fmm) {
        int rc = VP_OK;
        PROF(ctx, ST_FAR_FMM, s, rc = fmm_far(ctx, nf, f_dev, d, u_dev, qbuf, s));
        if (rc) {
            if (!profile) ctx->prof = prof_saved;
            return rc;
        }
    } else if (sym)
        PROF(ctx, ST_FAR_FF, s, launch_far_sym(ctx, nf, mesh->d_W, f_dev, u_dev, qbuf, s, f2out));
    else
        PROF(ctx, ST_FAR_FF, s,
             launch_far_ff(nf->src_ff, mesh->d_W, N, f_dev, d, nf->tgt_ff, nf->d_tnode, M, partial, qbuf, splits, s,
                           f2out, mesh->nq));
    if (splits > 1) PROF(ctx, ST_REDUCE, s, launch_reduce_splits(partial, splits, (int64_t)d * M, u_dev, s));
    if (precision == VP_MIXED_TC) {
        int rc = VP_OK;
        PROF(ctx, ST_APPLY_TC, s, rc = tc_apply(ctx, nf, f_dev, d, u_dev, apply_ws, s));
        if (rc) {
            if (!profile) ctx->prof = prof_saved;
            return rc;
        }
    } else if (mesh->rule.builtin < 0) {   // generated far rules: the FP64 apply for any node count
        PROF(ctx, ST_APPLY, s, launch_apply_fp64(nf->d_row, nf->d_ptri, nf->d_C, mesh->nq, f_dev, N, d, M, u_dev, fT, s));
    } else if ((precision == VP_MIXED || fmm) && d == 1 && nf->d_C2) {
        PROF(ctx, ST_APPLY, s,
             launch_apply_stream(nf->d_row, nf->d_ptri, nf->d_ptgt, nf->d_C2, mesh->nq, f_dev, N, nf->P, M, u_dev,
                                 apply_ws, ctx->d_flag, ctx->sm_count, s, f2out != nullptr));
    } else if ((precision == VP_MIXED || fmm) && d < APPLY_MANY_MIN_D && nf->d_C2) {
        PROF(ctx, ST_APPLY, s,
             launch_apply_f2(nf->d_row, nf->d_ptri, nf->d_C2, mesh->nq, f_dev, N, d, M, u_dev, (float2*)apply_ws, s));
    } else {
        PROF(ctx, ST_APPLY, s, launch_apply_fp64(nf->d_row, nf->d_ptri, nf->d_C, mesh->nq, f_dev, N, d, M, u_dev, fT, s));
    }
    if (!profile) ctx->prof = prof_saved;
    VP_LAUNCH_CHECK(ctx);
    return VP_OK;
}

extern "C" {

int vp_potential_eval(vp_ctx* ctx, const vp_nf* nf, const double* f_dev, int32_t d, double* u_dev, int32_t precision,
                      void* stream) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!nf_ok(nf) || nf->ctx != ctx) return vp_set_error(ctx, VP_ERR_STATE, "vp_potential_eval: bad near-field handle");
    if (!f_dev || !u_dev || d < 1 || d > 256 || precision < VP_FP64 || precision > VP_MIXED_FMM)
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_potential_eval: bad arguments");
    DevGuard g(ctx->device);
    if (precision == VP_MIXED_TC && !nf->tc) {
        int rc = tc_plan_build(ctx, const_cast<vp_nf*>(nf), 5, (cudaStream_t)stream);
        if (rc) return rc;
    }
    if (precision == VP_MIXED_FMM && !nf->fmm) {
        int rc = fmm_plan_build(ctx, const_cast<vp_nf*>(nf), (cudaStream_t)stream);
        if (rc) return rc;
    }
    if ((precision == VP_MIXED || precision == VP_MIXED_TC) && far_sym_applicable(nf, d) && !nf->sym) {
        int rc = far_sym_plan(ctx, const_cast<vp_nf*>(nf));
        if (rc) return rc;
    }

    int rc = ensure_ws(ctx, eval_ws_bytes(ctx, nf, d, precision));
    if (rc) return rc;
    return eval_impl(ctx, nf, f_dev, d, u_dev, precision, (cudaStream_t)stream, ctx->ws, true);
}

int vp_potential_eval_host(vp_ctx* ctx, const vp_nf* nf, const double* f_host, int32_t d, double* u_host,
                           int32_t precision, void* stream) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!nf_ok(nf) || nf->ctx != ctx) return vp_set_error(ctx, VP_ERR_STATE, "vp_potential_eval_host: bad handle");
    if (!f_host || !u_host || d < 1 || d > 256) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_potential_eval_host: bad arguments");
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = nf->mesh->N, M = nf->M;
    const size_t fb = (size_t)d * N * sizeof(double), ub = (size_t)d * M * sizeof(double);
    if (fb + ub > ctx->stage_bytes) {
        if (ctx->stage) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
        }
        VP_CUDA_TRY(ctx, cudaMalloc(&ctx->stage, fb + ub));
        ctx->stage_bytes = fb + ub;
    }
    double* fd = ctx->stage;
    double* ud = (double*)((char*)ctx->stage + fb);
    VP_CUDA_TRY(ctx, cudaMemcpyAsync(fd, f_host, fb, cudaMemcpyHostToDevice, s));
    int rc = vp_potential_eval(ctx, nf, fd, d, ud, precision, stream);
    if (rc) return rc;
    VP_CUDA_TRY(ctx, cudaMemcpyAsync(u_host, ud, ub, cudaMemcpyDeviceToHost, s));
    VP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return VP_OK;
}

int vp_nf_prepare_tc(vp_ctx* ctx, vp_nf* nf, int32_t levels, void* stream) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!nf_ok(nf) || nf->ctx != ctx) return vp_set_error(ctx, VP_ERR_STATE, "vp_nf_prepare_tc: bad near-field handle");
    DevGuard g(ctx->device);
    return tc_plan_build(ctx, nf, levels, (cudaStream_t)stream);
}

int vp_device_status(vp_ctx* ctx, void* stream) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_flag(ctx, ctx->d_flag, s);
    VP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int32_t), s));
    VP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return rc;
}

int vp_nf_fmm_info(const vp_nf* nf, int32_t* leaf_level, int64_t* n_boxes) {
    if (!nf_ok(nf)) return VP_ERR_STATE;
    if (leaf_level) *leaf_level = fmm_level(nf);
    if (n_boxes) *n_boxes = fmm_boxes(nf);
    return VP_OK;
}

int vp_nf_tc_info(const vp_nf* nf, int32_t* levels, int64_t* n_tiles, int64_t* n_chunks, int64_t* bytes) {
    if (!nf_ok(nf)) return VP_ERR_STATE;
    const TcPlan* p = nf->tc;
    if (levels) *levels = p ? p->levels : 0;
    if (n_tiles) *n_tiles = p ? p->n_tiles : 0;
    if (n_chunks) *n_chunks = p ? p->n_chunks : 0;
    if (bytes) *bytes = p ? (int64_t)p->bytes : 0;
    return VP_OK;
}

int vp_profile_enable(vp_ctx* ctx, int32_t on) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    ctx->prof = on != 0;
    return VP_OK;
}

int vp_profile_reset(vp_ctx* ctx) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    DevGuard g(ctx->device);
    prof_collect(ctx);
    for (int i = 0; i < ST_COUNT; i++) {
        ctx->prof_ms[i] = 0;
        ctx->prof_n[i] = 0;
    }
    return VP_OK;
}

int vp_profile_read(vp_ctx* ctx, char* names, int64_t* counts, double* ms, int32_t cap, int32_t* n) {
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    DevGuard g(ctx->device);
    prof_collect(ctx);
    if (n) *n = ST_COUNT;
    for (int i = 0; i < ST_COUNT && i < cap; i++) {
        if (names) {
            std::memset(names + 32 * i, 0, 32);
            std::strncpy(names + 32 * i, kStageNames[i], 31);
        }
        if (counts) counts[i] = ctx->prof_n[i];
        if (ms) ms[i] = ctx->prof_ms[i];
    }
    return VP_OK;
}

// ---------------------------------------------------------- interpolation
}  // extern "C"

namespace {

// Reference interpolation nodes of order N (the Blyth-Pozrikidis
// construction on the N + 1 Gauss-Legendre points) and the inverse of their
// Koornwinder interpolation matrix, in long double on the host.
void interp_reference(int N, std::vector<double>& zx, std::vector<double>& zy, std::vector<double>& Vinv) {
    typedef long double LD;
    const int n1 = N + 1;
    // Gauss-Legendre points: Newton on P_{n1} from Chebyshev-like guesses
    std::vector<LD> g(n1);
    const LD pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n1; i++) {
        LD x = std::cos(pi * (i + 0.75L) / (n1 + 0.5L));
        for (int it = 0; it < 100; it++) {
            LD p0 = 1.0L, p1 = x;
            for (int k = 1; k < n1; k++) {
                const LD p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
                p0 = p1;
                p1 = p2;
            }
            const LD dp = n1 * (x * p1 - p0) / (x * x - 1.0L);
            const LD dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-30L) break;
        }
        g[i] = x;
    }
    std::sort(g.begin(), g.end());
    std::vector<LD> v(n1);
    for (int i = 0; i < n1; i++) v[i] = 0.5L * (g[i] + 1.0L);
    const int nn = (N + 1) * (N + 2) / 2;
    std::vector<LD> X, Y;
    for (int j = 0; j <= N; j++)
        for (int i = 0; i <= N - j; i++) {
            const int k = N - i - j;
            X.push_back((1.0L + 2.0L * v[i] - v[j] - v[k]) / 3.0L);
            Y.push_back((1.0L + 2.0L * v[j] - v[i] - v[k]) / 3.0L);
        }
    // interpolation matrix A[i][a] = K_a(node i) (Section 2.1)
    std::vector<LD> A((size_t)nn * nn);
    for (int r = 0; r < nn; r++) {
        const LD x = X[r], y = Y[r], w = 1.0L - x, s = 2.0L * y - w, z = 2.0L * x - 1.0L;
        std::vector<LD> H(N + 2);
        H[0] = 1.0L;
        H[1] = s;
        for (int m = 1; m < N; m++) H[m + 1] = ((2 * m + 1) * s * H[m] - m * w * w * H[m - 1]) / (m + 1);
        for (int m = 0; m <= N; m++) {
            const LD a = 2.0L * m + 1.0L;
            LD pkm1 = 0.0L, pk = 1.0L;
            for (int k = 0; k <= N - m; k++) {
                const int n = m + k;
                A[(size_t)r * nn + n * (n + 1) / 2 + m] = std::sqrt(2.0L * a * (n + 1)) * H[m] * pk;
                LD pn;
                if (k == 0) pn = 0.5L * ((a + 2.0L) * z + a);
                else {
                    const LD c1 = 2.0L * k + a;
                    pn = ((c1 + 1.0L) * ((c1 + 2.0L) * c1 * z + a * a) * pk - 2.0L * k * (k + a) * (c1 + 2.0L) * pkm1) /
                         (2.0L * (k + 1.0L) * (k + a + 1.0L) * c1);
                }
                pkm1 = pk;
                pk = pn;
            }
        }
    }
    // Gauss-Jordan with partial pivoting: [A | I] -> [I | A^-1]
    std::vector<LD> B((size_t)nn * nn, 0.0L);
    for (int i = 0; i < nn; i++) B[(size_t)i * nn + i] = 1.0L;
    for (int c = 0; c < nn; c++) {
        int piv = c;
        for (int r = c + 1; r < nn; r++)
            if (std::fabs(A[(size_t)r * nn + c]) > std::fabs(A[(size_t)piv * nn + c])) piv = r;
        if (piv != c)
            for (int k = 0; k < nn; k++) {
                std::swap(A[(size_t)c * nn + k], A[(size_t)piv * nn + k]);
                std::swap(B[(size_t)c * nn + k], B[(size_t)piv * nn + k]);
            }
        const LD d = A[(size_t)c * nn + c];
        for (int k = 0; k < nn; k++) {
            A[(size_t)c * nn + k] /= d;
            B[(size_t)c * nn + k] /= d;
        }
        for (int r = 0; r < nn; r++) {
            if (r == c) continue;
            const LD f = A[(size_t)r * nn + c];
            if (f == 0.0L) continue;
            for (int k = 0; k < nn; k++) {
                A[(size_t)r * nn + k] -= f * A[(size_t)c * nn + k];
                B[(size_t)r * nn + k] -= f * B[(size_t)c * nn + k];
            }
        }
    }
    // coefficients = A^-1 u: row a of A^-1 (basis a) against node values
    zx.resize(nn);
    zy.resize(nn);
    Vinv.resize((size_t)nn * nn);
    for (int i = 0; i < nn; i++) {
        zx[i] = (double)X[i];
        zy[i] = (double)Y[i];
    }
    for (size_t i = 0; i < (size_t)nn * nn; i++) Vinv[i] = (double)B[i];
}

// Recurrence table of the device's Koornwinder sums (k_interp.cu), for
// degree N with nn = dim P_N entries per array, index a = n (n + 1)/2 + m:
// [c_mn][jA][jB][jC] (the Jacobi coefficients that advance P_{n-m}^{(2m+1,0)}
// to degree n - m + 1, stored at a) then hA[m], hB[m], m = 0..N.
void interp_recurrences(int N, std::vector<double>& rec) {
    typedef long double LD;
    const int nn = (N + 1) * (N + 2) / 2;
    rec.assign(4 * nn + 2 * (N + 1), 0.0);
    for (int m = 0; m <= N; m++) {
        const LD al = 2.0L * m + 1.0L;
        for (int n = m; n <= N; n++) {
            const int a = n * (n + 1) / 2 + m, k = n - m;
            rec[a] = (double)std::sqrt(2.0L * al * (n + 1));
            LD A, B, Cc;
            if (k == 0) {
                A = 0.5L * (al + 2.0L);
                B = 0.5L * al;
                Cc = 0.0L;
            } else {
                const LD c1 = 2.0L * k + al, den = 2.0L * (k + 1) * (k + al + 1) * c1;
                A = (c1 + 1.0L) * (c1 + 2.0L) * c1 / den;
                B = (c1 + 1.0L) * al * al / den;
                Cc = 2.0L * k * (k + al) * (c1 + 2.0L) / den;
            }
            rec[nn + a] = (double)A;
            rec[2 * nn + a] = (double)B;
            rec[3 * nn + a] = (double)Cc;
        }
        rec[4 * nn + m] = (double)((2.0L * m + 1.0L) / (m + 1.0L));
        rec[4 * nn + (N + 1) + m] = (double)((LD)m / (m + 1.0L));
    }
}

}  // namespace

struct vp_interp {
    vp_ctx* ctx = nullptr;
    vp_mesh* mesh = nullptr;       // the interpolation mesh (its own quadrature nodes are unused)
    int N = 0, nn = 0;
    double* d_zx = nullptr;        // [nn] reference nodes
    double* d_zy = nullptr;
    double* d_Vinv = nullptr;      // [nn][nn] basis x node
    double* d_rec = nullptr;       // Koornwinder recurrence table (interp_recurrences)
    int64_t* d_cell_start = nullptr;
    int32_t* d_cell_tri = nullptr;
    GridDev g{};
    int magic = 0x56504950;
};

static bool interp_ok(const vp_interp* p) { return p && p->magic == 0x56504950; }

static void interp_free(vp_interp* p) {
    void* ps[] = {p->d_zx, p->d_zy, p->d_Vinv, p->d_rec, p->d_cell_start, p->d_cell_tri};
    for (void* q : ps)
        if (q) cudaFree(q);
    if (p->mesh) vp_mesh_release(p->mesh);
    p->magic = 0;
    delete p;
}

extern "C" {

int vp_interp_create(vp_ctx* ctx, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* cidx,
                     const double* coef, int64_t ncurve, int32_t K, int32_t order, void* stream, vp_interp** out) {
    if (out) *out = nullptr;
    if (!ctx_ok(ctx)) return VP_ERR_STATE;
    if (!out || order < 1 || order > 20) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_interp_create: bad arguments");
    vp_interp* ip = new (std::nothrow) vp_interp();
    if (!ip) return VP_ERR_OOM;
    ip->ctx = ctx;
    ip->N = order;
    ip->nn = (order + 1) * (order + 2) / 2;
    int rc = cidx ? vp_mesh_upload_curved(ctx, vxy, nv, tri, nt, cidx, coef, ncurve, K, VP_RULE_16_D8, stream, &ip->mesh)
                  : vp_mesh_upload(ctx, vxy, nv, tri, nt, VP_RULE_16_D8, stream, &ip->mesh);
    if (rc) {
        delete ip;
        return rc;
    }
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> zx, zy, Vinv, rec;
    interp_reference(order, zx, zy, Vinv);
    interp_recurrences(order, rec);
    const int nn = ip->nn;
#define IP_FAIL(code, msg)                     \
    do {                                       \
        rc = vp_set_error(ctx, (code), (msg)); \
        interp_free(ip);                       \
        return rc;                             \
    } while (0)
    if (dev_alloc(&ip->d_zx, nn) != cudaSuccess || dev_alloc(&ip->d_zy, nn) != cudaSuccess ||
        dev_alloc(&ip->d_Vinv, (size_t)nn * nn) != cudaSuccess || dev_alloc(&ip->d_rec, rec.size()) != cudaSuccess)
        IP_FAIL(VP_ERR_OOM, "vp_interp_create: device allocation failed");
    if (cudaMemcpyAsync(ip->d_rec, rec.data(), rec.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        IP_FAIL(VP_ERR_CUDA, "vp_interp_create: copy failed");
    if (cudaMemcpyAsync(ip->d_zx, zx.data(), nn * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ip->d_zy, zy.data(), nn * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ip->d_Vinv, Vinv.data(), (size_t)nn * nn * sizeof(double), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        IP_FAIL(VP_ERR_CUDA, "vp_interp_create: copy failed");
    // grid of element boxes for point location
    {
        const vp_mesh* m = ip->mesh;
        Scratch sc(s);
        double *d_bbox, *d_red;
        int32_t *d_cnt, *d_max;
        int64_t* d_cursor;
        if (sc.alloc(&d_bbox, 4 * nt) != cudaSuccess || sc.alloc(&d_red, 4) != cudaSuccess)
            IP_FAIL(VP_ERR_OOM, "vp_interp_create: device allocation failed");
        launch_tri_bbox(m->d_tv, nt, d_bbox, s);
        if (m->d_cidx) launch_curved_bbox(nt, mesh_curves(m), d_bbox, s);
        launch_bbox_reduce(d_bbox, nt, 4, d_red, s);
        std::vector<double> hb(4 * nt);
        double h_red[4];
        if (cudaMemcpyAsync(hb.data(), d_bbox, 4 * nt * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(h_red, d_red, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            IP_FAIL(VP_ERR_CUDA, "vp_interp_create: box copy failed");
        // cell = the median element box size
        std::vector<double> sizes(nt);
        for (int64_t t = 0; t < nt; t++) sizes[t] = std::max(hb[4 * t + 2] - hb[4 * t], hb[4 * t + 3] - hb[4 * t + 1]);
        std::nth_element(sizes.begin(), sizes.begin() + nt / 2, sizes.end());
        const double W_ = h_red[2] - h_red[0], H_ = h_red[3] - h_red[1];
        double hc = std::max(sizes[nt / 2], std::max(W_, H_) / 4096.0);
        hc = std::max(hc, 1e-300);
        int64_t nx = std::max<int64_t>(1, (int64_t)std::ceil(W_ / hc)), ny = std::max<int64_t>(1, (int64_t)std::ceil(H_ / hc));
        while (nx * ny > ((int64_t)1 << 24)) {
            hc *= 1.5;
            nx = std::max<int64_t>(1, (int64_t)std::ceil(W_ / hc));
            ny = std::max<int64_t>(1, (int64_t)std::ceil(H_ / hc));
        }
        const int64_t ncell = nx * ny;
        GridDev gd;
        gd.ox = h_red[0];
        gd.oy = h_red[1];
        gd.h = hc;
        gd.nx = (int32_t)nx;
        gd.ny = (int32_t)ny;
        gd.cell_start = nullptr;
        gd.cell_tri = nullptr;
        int64_t nentries = 0;
        int32_t h_max = 0;
        if (sc.alloc(&d_cnt, ncell) != cudaSuccess || sc.alloc(&d_cursor, ncell + 1) != cudaSuccess ||
            sc.alloc(&d_max, 1) != cudaSuccess || dev_alloc(&ip->d_cell_start, ncell + 1) != cudaSuccess)
            IP_FAIL(VP_ERR_OOM, "vp_interp_create: device allocation failed");
        cudaMemsetAsync(d_cnt, 0, ncell * sizeof(int32_t), s);
        launch_tri_cell_count(d_bbox, nt, gd, d_cnt, s);
        rc = vp_exclusive_scan_i32(ctx, d_cnt, ip->d_cell_start, ncell, s);
        if (rc) {
            interp_free(ip);
            return rc;
        }
        launch_max_i32(d_cnt, ncell, d_max, s);
        if (cudaMemcpyAsync(&nentries, ip->d_cell_start + ncell, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(&h_max, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            IP_FAIL(VP_ERR_CUDA, "vp_interp_create: grid count failed");
        if (h_max > 16384) IP_FAIL(VP_ERR_CUDA, "vp_interp_create: a grid cell holds more than 16384 elements");
        if (dev_alloc(&ip->d_cell_tri, std::max<int64_t>(1, nentries)) != cudaSuccess)
            IP_FAIL(VP_ERR_OOM, "vp_interp_create: device allocation failed");
        cudaMemcpyAsync(d_cursor, ip->d_cell_start, (ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        launch_tri_cell_fill(d_bbox, nt, gd, d_cursor, ip->d_cell_tri, s);
        gd.cell_start = ip->d_cell_start;
        gd.cell_tri = ip->d_cell_tri;
        cudaMemsetAsync(ctx->d_flag, 0, sizeof(int32_t), s);
        launch_cell_sort(gd, ncell, h_max, ip->d_cell_tri, ctx->d_flag, s);
        if (cudaGetLastError() != cudaSuccess) IP_FAIL(VP_ERR_CUDA, "vp_interp_create: grid build failed");
        rc = check_flag(ctx, ctx->d_flag, s);
        if (rc) {
            interp_free(ip);
            return rc;
        }
        ip->g = gd;
    }
#undef IP_FAIL
    *out = ip;
    return VP_OK;
}

int vp_interp_info(const vp_interp* ip, int64_t* n_tri, int64_t* n_nodes, int32_t* nodes_per_tri) {
    if (!interp_ok(ip)) return VP_ERR_STATE;
    if (n_tri) *n_tri = ip->mesh->nt;
    if (n_nodes) *n_nodes = ip->mesh->nt * ip->nn;
    if (nodes_per_tri) *nodes_per_tri = ip->nn;
    return VP_OK;
}

int vp_interp_nodes(const vp_interp* ip, double* xy_dev, void* stream) {
    if (!interp_ok(ip)) return VP_ERR_STATE;
    if (!xy_dev) return vp_set_error(ip->ctx, VP_ERR_INVALID_ARG, "vp_interp_nodes: bad arguments");
    DevGuard g(ip->ctx->device);
    launch_interp_nodes(ip->mesh->d_tv, mesh_curves(ip->mesh), ip->mesh->nt, ip->d_zx, ip->d_zy, ip->nn, xy_dev,
                        (cudaStream_t)stream);
    VP_LAUNCH_CHECK(ip->ctx);
    return VP_OK;
}

int vp_interp_coeffs(vp_interp* ip, const double* u_dev, int32_t d, double* coef_dev, void* stream) {
    if (!interp_ok(ip)) return VP_ERR_STATE;
    if (!u_dev || !coef_dev || d < 1 || d > 65535)
        return vp_set_error(ip->ctx, VP_ERR_INVALID_ARG, "vp_interp_coeffs: bad arguments");
    DevGuard g(ip->ctx->device);
    launch_interp_coeffs(ip->d_Vinv, ip->nn, ip->mesh->nt, d, u_dev, coef_dev, (cudaStream_t)stream);
    VP_LAUNCH_CHECK(ip->ctx);
    return VP_OK;
}

int vp_interp_eval(vp_interp* ip, const double* coef_dev, int32_t d, const double* pts_dev, int64_t m,
                   double* out_dev, int32_t* elem_dev, void* stream) {
    if (!interp_ok(ip)) return VP_ERR_STATE;
    if (!coef_dev || d < 1 || m < 0 || (m > 0 && (!pts_dev || !out_dev)))
        return vp_set_error(ip->ctx, VP_ERR_INVALID_ARG, "vp_interp_eval: bad arguments");
    DevGuard g(ip->ctx->device);
    launch_interp_eval(ip->mesh->d_tv, mesh_curves(ip->mesh), ip->g, pts_dev, m, ip->N, ip->nn, ip->mesh->nt,
                       ip->d_rec, coef_dev, d, out_dev, elem_dev, (cudaStream_t)stream);
    VP_LAUNCH_CHECK(ip->ctx);
    return VP_OK;
}

void vp_interp_release(vp_interp* ip) {
    if (!interp_ok(ip)) return;
    DevGuard g(ip->ctx->device);
    cudaDeviceSynchronize();
    interp_free(ip);
}

int vp_rule_table(int32_t which, double* x, double* y, double* w, double* what, int32_t cap, int32_t* n) {
    const double *X = nullptr, *Y = nullptr, *Wt = nullptr;
    double wh = 0.0;
    int32_t len = 0;
    switch (which) {
        case 16: X = VP_FAR16_X; Y = VP_FAR16_Y; Wt = VP_FAR16_W; wh = VP_FAR16_WHAT; len = 16; break;
        case 19: X = VP_FAR19_X; Y = VP_FAR19_Y; Wt = VP_FAR19_W; wh = VP_FAR19_WHAT; len = 19; break;
        case 33: X = VP_NEAR33_X; Y = VP_NEAR33_Y; Wt = VP_NEAR33_W; wh = VP_NEAR33_WHAT; len = 33; break;
        case 8: X = VP_GGQ8_R; Wt = VP_GGQ8_W; len = 8; break;
        case 5: X = VP_RAD5_R; Y = VP_RAD5_B; Wt = VP_RAD5_A; len = 5; break;
        case 116: X = VP_GL16_X; Wt = VP_GL16_W; len = 16; break;
        default: return VP_ERR_INVALID_ARG;
    }
    if (n) *n = len;
    if (cap < len) return VP_ERR_INVALID_ARG;
    for (int32_t i = 0; i < len; i++) {
        if (x) x[i] = X[i];
        if (y) y[i] = Y ? Y[i] : 0.0;
        if (w) w[i] = Wt[i];
    }
    if (what) *what = wh;
    return VP_OK;
}

}  // extern "C"
