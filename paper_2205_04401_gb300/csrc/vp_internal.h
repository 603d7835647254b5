// Internal structures of libvp (host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/vp.h"
#include "vp_device.cuh"
#include "vp_curved.cuh"

// Far-field source/target coordinates in float-float: value = hi + lo, with
// hi on a fixed dyadic grid of spacing q so that hi_t - hi_s is exact in FP32.
struct FFCoords {
    float* hi = nullptr;  // [n][2]
    float* lo = nullptr;  // [n][2]
};

enum VpStage {
    ST_MESH_NODES = 0, ST_TRI_GEOM, ST_TRI_CELLS, ST_CELL_SORT, ST_TARGET_CELLS, ST_LOCATE, ST_LIST_COUNT,
    ST_LIST_FILL, ST_WEIGHTS_SELF, ST_WEIGHTS_NEAR, ST_FF_SPLIT, ST_FAR_FP64, ST_FAR_FF, ST_REDUCE, ST_APPLY,
    ST_APPLY_TC, ST_WEIGHTS_CURVED, ST_FAR_FMM, ST_COUNT
};

// A far rule on the device: reference nodes and weights and the map Q from
// the P_4 moments of a pair to its nodal correction weights (vp_rules.cu).
struct FarRuleDev {
    const double* x = nullptr;    // [nq]
    const double* y = nullptr;    // [nq]
    const double* w = nullptr;    // [nq]
    const double* Q = nullptr;    // [nq][VP_NB], moments in the tensor-Legendre basis (leg15)
    const float2* Q2 = nullptr;   // [nq][VP_NB], float-float, moments in the monomial basis (f2_mon15_acc)
    const float2* B2 = nullptr;   // [VP_NNEAR][nq], float-float: root-leaf map, C_k = sum_j B2[j nq + k] g_j
    int nq = 0;
};
struct FarRule {
    FarRuleDev dev;
    double what = 0.0;      // w-hat of Eq. rho0
    int degree = 0;         // total degree N_f
    int code = 0;           // vp_rule value
    int builtin = -1;       // index into VpTables (0: 16 nodes, 1: 19 nodes), -1 generated
    void* d_buf = nullptr;  // generated rules: device block owned by the context
};

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

struct vp_ctx {
    int device = 0;
    int sm_count = 0;
    std::string last_error;
    VpTables* d_tables = nullptr;
    VpTables h_tables;
    int32_t* d_flag = nullptr;     // device error flags (one int)
    // evaluation workspace (grown on demand)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // staging for the host-buffer entry point
    double* stage = nullptr;
    size_t stage_bytes = 0;
    // profiling (see vp_profile_enable)
    bool prof = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[ST_COUNT] = {0};
    int ff_tpt[4] = {0, 0, 0, 0};   // autotuned targets per thread of the batched far sum, per chunk width
    int ff_tpt_fixed[4] = {0, 0, 0, 0};   // vp_set_batch_tile: fixed targets per thread (0: autotune)
    int64_t far_sym_cap_bytes = int64_t(256) << 20;   // column scratch per band of the symmetric far sum
    int64_t prof_n[ST_COUNT] = {0};
    // generated far rules, made on first use and kept until vp_destroy
    std::vector<FarRule> gen_rules;
    std::mutex rule_mu;
    int magic = 0x56504358;
};

// far rules (vp_rules.cu)
bool far_rule_valid(int32_t rule);
// B2[j nq + k] = sum_i QM[k][i] M_i(u_j, v_j) at the near-rule nodes (float-float)
void root_leaf_map(const double* QM, int nq, float2* B2);
int far_rule_nq(int32_t rule);
int far_rule_get(vp_ctx* ctx, int32_t rule, FarRule* out);
void far_rules_free(vp_ctx* ctx);

// Stage timing helpers (no-ops unless profiling is enabled).
void prof_begin(vp_ctx* ctx, int stage, cudaStream_t s, ProfRec& r);
void prof_end(vp_ctx* ctx, cudaStream_t s, ProfRec& r);
void prof_collect(vp_ctx* ctx);

// Run the statements between the events of a profiled stage.
#define PROF(ctx, stage, s, ...)        \
    do {                                \
        ProfRec _r;                     \
        prof_begin(ctx, stage, s, _r);  \
        __VA_ARGS__;                    \
        prof_end(ctx, s, _r);           \
    } while (0)

struct vp_mesh {
    vp_ctx* ctx = nullptr;
    int64_t nt = 0, nv = 0, N = 0;
    int nq = 0;
    FarRule rule;                // far rule of the nodes (Section 3.2)
    double* d_tv = nullptr;      // [nt][6] counter-clockwise vertex coordinates
    double* d_J = nullptr;       // [nt] J_T = 2 area
    double* d_y = nullptr;       // [N][2]
    double* d_W = nullptr;       // [N]
    double bbox[4] = {0, 0, 0, 0};   // of the vertices and, with curves, of the curved sides
    // curved elements (vp_mesh_upload_curved): curve of each triangle (-1
    // straight) and Chebyshev coefficients [ncurve][2][K+1]; nullptr if none
    int32_t* d_cidx = nullptr;
    double* d_coef = nullptr;
    double* d_dcoef = nullptr;     // Chebyshev coefficients of dD/dt, same layout
    int64_t ncurve = 0;
    int K = 0;
    int magic = 0x56504d48;
};

// Tensor-core correction apply: the correction matrix re-laid per tile of 128
// targets (Morton order) as dense bf16 digit images over the union of the
// tile's triangles (k_tc.cu).
struct TcPlan {
    int levels = 0;                 // digits per value
    int64_t n_tiles = 0, n_chunks = 0;
    int32_t* d_perm = nullptr;      // [n_tiles 128] targets of each tile (-1 pads)
    int32_t* d_pos = nullptr;       // [M] position of each target in d_perm
    int64_t* d_chunk_ptr = nullptr; // [n_tiles + 1] first chunk of each tile
    int32_t* d_chunk_near = nullptr;// [n_tiles] near-pair chunks of each tile (its self chunks follow)
    int32_t* d_chunk_tri = nullptr; // [n_chunks][2] triangles of each chunk
    int32_t* d_rexp = nullptr;      // [2][M] row exponents of the near and the self weights
    uint32_t* d_gmask = nullptr;    // [n_chunks] row groups (8 targets) with weights in the chunk
    int64_t* d_gptr = nullptr;      // [n_chunks + 1] first stored row group of each chunk
    uint16_t* d_A = nullptr;        // [stored row groups] digit images (bf16 bits)
    int64_t n_groups = 0;           // stored row groups
    size_t a_bytes = 0, bytes = 0;
};

struct SymPlan;   // symmetric far-sum work units (k_far_sym.cu)
struct FmmPlan;   // quadtree, sorted sources and targets, translation tables (k_fmm.cu)

struct vp_nf {
    vp_ctx* ctx = nullptr;
    const vp_mesh* mesh = nullptr;
    int64_t M = 0, P = 0, n_extra = 0;
    int node_targets = 0;
    vp_nf_params params{};
    double* d_txy = nullptr;      // [M][2]
    int32_t* d_tself = nullptr;   // [M]
    int32_t* d_tnode = nullptr;   // [M]
    int64_t* d_row = nullptr;     // [M+1]
    int32_t* d_ptri = nullptr;    // [P]
    int32_t* d_ptgt = nullptr;    // [P]
    uint8_t* d_pkind = nullptr;   // [P]
    double* d_C = nullptr;        // [P][nq]
    float2* d_C2 = nullptr;       // [P][nq] the same weights as float-float pairs (float-float builds)
    FFCoords src_ff, tgt_ff;      // float-float copies for the mixed far sum
    double ff_origin[2] = {0, 0};
    double ff_scale = 1.0;         // grid spacing q of the hi parts
    vp_nf_stats_t stats{};
    TcPlan* tc = nullptr;          // tensor-core apply plan (vp_nf_prepare_tc)
    SymPlan* sym = nullptr;        // symmetric far sum over the node targets (built on first use)
    FmmPlan* fmm = nullptr;        // fast multipole far sum (VP_MIXED_FMM, built on first use)
    int magic = 0x56504e46;
};

// ----------------------------------------------------------- utilities
#define VP_CUDA_TRY(ctx, expr)                                                              \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            if (ctx) (ctx)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e); \
            return _e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA;              \
        }                                                                                   \
    } while (0)

// Launch-time error check (async errors are caught at the next sync).
#define VP_LAUNCH_CHECK(ctx) VP_CUDA_TRY(ctx, cudaGetLastError())

int vp_set_error(vp_ctx* ctx, int code, const std::string& msg);

// Per-unit device set-up run by vp_create with the context's device current:
// each float-float unit copies its log table (vp_ff.cuh), and the
// allocation-free evaluation resolves its fixed scratch array, so that no
// later call loads a module, copies a table or looks up a symbol.
cudaError_t eval_module_prepare();
cudaError_t far_sym_module_prepare();
cudaError_t batch_module_prepare();
cudaError_t fmm_module_prepare();
cudaError_t weights_module_prepare();
int noalloc_prepare(vp_ctx* ctx);

// Source splits of the one-sided far sum for M targets and N sources
// (blocks of `threads` targets, about four blocks per SM in all).
int eval_splits(const vp_ctx* ctx, int64_t M, int64_t N, int threads);

// Evaluation with explicit workspace (vp_potential_eval's body).
size_t eval_ws_bytes(const vp_ctx* ctx, const vp_nf* nf, int d, int precision);
int eval_impl(vp_ctx* ctx, const vp_nf* nf, const double* f_dev, int32_t d, double* u_dev, int32_t precision,
              cudaStream_t s, void* ws, bool profile);

// ----------------------------------------------------------- launchers
// scan: out[0] = 0, out[i+1] = sum_{j<=i} in[j] (int32 or int64 input), n >= 0
int vp_exclusive_scan_i32(vp_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
int vp_exclusive_scan_i64(vp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

// mesh
void launch_mesh_nodes(const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, FarRuleDev fr, double* tv,
                       double* J, double* y, double* W, int32_t* flag, cudaStream_t s);

// lists
struct GridDev {
    double ox, oy, h;
    int32_t nx, ny;
    const int64_t* cell_start;  // [ncell+1]
    const int32_t* cell_tri;    // sorted ascending per cell
};
void launch_tri_geom(const double* tv, const double* J, int64_t nt, double what, int N, double eps, double cn,
                     double* R, double* bbox, cudaStream_t s);
void launch_bbox_reduce(const double* bbox, int64_t n, int stride, double* out4, cudaStream_t s);
void launch_tri_cell_count(const double* bbox, int64_t nt, GridDev g, int32_t* cnt, cudaStream_t s);
void launch_tri_cell_fill(const double* bbox, int64_t nt, GridDev g, int64_t* cursor, int32_t* cell_tri,
                          cudaStream_t s);
void launch_cell_sort(GridDev g, int64_t ncell, int32_t max_count, int32_t* cell_tri, int32_t* flag,
                      cudaStream_t s);
void launch_max_i32(const int32_t* a, int64_t n, int32_t* out, cudaStream_t s);
void launch_targets_init(const double* ynode, int64_t N, int nq, int node_targets, const double* extra, int64_t m,
                         double* txy, int32_t* tnode, int32_t* tself, cudaStream_t s);
void launch_target_cells(const double* txy, int64_t M, GridDev g, int32_t* tcell, int32_t* cnt, cudaStream_t s);
void launch_target_order(const int32_t* tcell, int64_t M, int64_t* cursor, int32_t* order, cudaStream_t s);
void launch_locate(const double* tv, const double* txy, const int32_t* order, const int32_t* tcell, int64_t M,
                   GridDev g, int32_t* tself, cudaStream_t s);
void launch_list_pass(const double* tv, const double* R, int N, const double* txy, const int32_t* tself,
                      const int32_t* order, const int32_t* tcell, int64_t M, GridDev g, int32_t* count,
                      const int64_t* row, int32_t* ptri, int32_t* ptgt, uint8_t* pkind, uint32_t* cache, int cap,
                      cudaStream_t s);
void launch_split_pairs(const uint8_t* pkind, int64_t P, int32_t* near_idx, int32_t* self_idx,
                        unsigned long long* counters, cudaStream_t s);

// curved elements (k_curved.cu)
inline CurveDev mesh_curves(const vp_mesh* m) { return CurveDev{m->d_cidx, m->d_coef, m->d_dcoef, m->K}; }
void launch_mesh_nodes_curved(const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, CurveDev cv,
                              FarRuleDev fr, const double* tv, double* y, double* W, int32_t* flag, cudaStream_t s);
void launch_curved_bbox(int64_t nt, CurveDev cv, double* bbox, cudaStream_t s);
void launch_locate_curved(const double* tv, CurveDev cv, const double* txy, const int32_t* order,
                          const int32_t* tcell, int64_t M, GridDev g, int32_t* tself, cudaStream_t s);
// counters[0..3]: near straight, self straight, near curved, self curved
void launch_split_pairs4(const uint8_t* pkind, const int32_t* ptri, CurveDev cv, int64_t P, int32_t* near_idx,
                         int32_t* self_idx, int32_t* cnear_idx, int32_t* cself_idx, unsigned long long* counters,
                         cudaStream_t s);

// weights
struct WeightsArgs {
    const VpTables* tab;
    const double* Q;    // far rule's moment-to-weight map [nq][VP_NB] (tensor-Legendre moments)
    const float2* Q2;   // float-float map for monomial-basis moments (the float-float kernels)
    const float2* B2;   // root-leaf map of the far rule (k_weights_near_root)
    int nq;
    const double* tv;
    const double* J;
    const double* y;
    const double* W;
    const double* txy;
    const int32_t* tnode;
    const int32_t* ptri;
    const int32_t* ptgt;
    double* C;
    float2* C2;         // float-float copy of C (float-float kernels), or nullptr
    int32_t* pstat;     // per pair: leaves or panels
    int32_t* pcap;      // per pair: depth-capped leaves
    int32_t* flag;
    double eps, c_near;
    int depth_cap;
    int fp64;           // 1: node quadratures in FP64 (reference); 0: float-float
    int64_t nt, M, N;   // triangles, targets, nodes
    void* f2_ws;        // scratch of weights_f2_bytes(nt, M, N, n_near) for the float-float kernels
};
size_t weights_f2_bytes(int64_t nt, int64_t M, int64_t N, int64_t n_near);
// self and near weights (stages ST_WEIGHTS_SELF, ST_WEIGHTS_NEAR)
void launch_weights(const WeightsArgs& a, const int32_t* self_idx, int64_t n_self, const int32_t* near_idx,
                    int64_t n_near, cudaStream_t s, vp_ctx* ctx);
// interpolation over a mesh (k_interp.cu)
void launch_interp_nodes(const double* tv, CurveDev cv, int64_t nt, const double* zx, const double* zy, int nn,
                         double* xy, cudaStream_t s);
void launch_interp_coeffs(const double* Vinv, int nn, int64_t nt, int d, const double* u, double* coef,
                          cudaStream_t s);
void launch_tri_bbox(const double* tv, int64_t nt, double* bbox, cudaStream_t s);
// rec: the recurrence table of interp_recurrences (vp_api.cu)
void launch_interp_eval(const double* tv, CurveDev cv, GridDev g, const double* pts, int64_t m, int N, int nn,
                        int64_t nt, const double* rec, const double* coef, int d, double* out, int32_t* elem,
                        cudaStream_t s);
// correction weights of the pairs on curved triangles (stage ST_WEIGHTS_CURVED)
void launch_weights_curved(const WeightsArgs& a, CurveDev cv, const int32_t* self_idx, int64_t n_self,
                           const int32_t* near_idx, int64_t n_near, cudaStream_t s, vp_ctx* ctx);
void launch_sum_i32(const int32_t* a, int64_t n, unsigned long long* out, cudaStream_t s);
// out[0..2] = sums of a over kind 0 and kind != 0, sum of b
void launch_sum_by_kind(const int32_t* a, const uint8_t* kind, const int32_t* b, int64_t n, unsigned long long* out,
                        cudaStream_t s);

// evaluation
void launch_far_fp64(const double* y, const double* W, int64_t N, const double* f, int d, const double* txy,
                     const int32_t* tnode, int64_t M, double* partial, int splits, cudaStream_t s);
// f2out (d = 1 only, may be nullptr): also write the density as float-float
// pairs for the streamed correction apply (fused into the charge preparation)
void launch_far_ff(const FFCoords& src, const double* W, int64_t N, const double* f, int d, const FFCoords& tgt,
                   const int32_t* tnode, int64_t M, double* partial, float* qbuf, int splits, cudaStream_t s,
                   float2* f2out = nullptr, int nq = 1);
void launch_reduce_splits(const double* partial, int splits, int64_t count, double* out, cudaStream_t s);
// Densities from which the correction is applied with densities across lanes
// (needs a node-major copy of f: apply_ws_bytes); fewer, or fT == nullptr,
// take the entry-parallel kernel that needs no workspace.
constexpr int APPLY_MANY_MIN_D = 16;
size_t apply_ws_bytes(int64_t N, int d);
void launch_apply_fp64(const int64_t* row, const int32_t* ptri, const double* C, int nq, const double* f, int64_t N,
                       int d, int64_t M, double* u, double* fT, cudaStream_t s);
// symmetric far sum (k_far_sym.cu): one density, node targets first, N large
bool far_sym_applicable(const vp_nf* nf, int d);
int far_sym_plan(vp_ctx* ctx, vp_nf* nf);
void far_sym_plan_free(SymPlan* p);
size_t far_sym_ws_bytes(const vp_ctx* ctx, const vp_nf* nf);
void launch_far_sym(const vp_ctx* ctx, const vp_nf* nf, const double* W, const double* f, double* out, void* ws,
                    cudaStream_t s, float2* f2out = nullptr);

// fast multipole far sum (k_fmm.cu): plan on first use, workspace, evaluation
// (writes u = far sum, d densities), leaf level of a plan
int fmm_plan_build(vp_ctx* ctx, vp_nf* nf, cudaStream_t s);
void fmm_plan_free(FmmPlan* p);
size_t fmm_ws_bytes(const vp_nf* nf, int d);
int fmm_far(vp_ctx* ctx, const vp_nf* nf, const double* f, int d, double* u, void* ws, cudaStream_t s);
int fmm_level(const vp_nf* nf);
int64_t fmm_boxes(const vp_nf* nf);

// tensor-core apply (k_tc.cu)
int tc_plan_build(vp_ctx* ctx, vp_nf* nf, int levels, cudaStream_t s);
void tc_plan_free(TcPlan* p);
size_t tc_ws_bytes(const vp_nf* nf);
int tc_apply(vp_ctx* ctx, const vp_nf* nf, const double* f, int d, double* u, void* ws, cudaStream_t s);
void launch_ff_split(const double* xy, int64_t n, double ox, double oy, double q, FFCoords out, cudaStream_t s);
// float-float copies and the float-float apply of the mixed path (d < APPLY_MANY_MIN_D)
void launch_to_f2(const double* x, int64_t n, float2* out, cudaStream_t s);
void launch_apply_f2(const int64_t* row, const int32_t* ptri, const float2* C2, int nq, const double* f, int64_t N,
                     int d, int64_t M, double* u, float2* f2v, cudaStream_t s);
// streamed float-float apply of one density (k_apply_stream.cu), workspace of
// apply_stream_ws_bytes(N, P); ptri, ptgt and C2 carry 16 bytes of padding
size_t apply_stream_ws_bytes(int64_t N, int64_t P);
// The float-float density the streamed apply gathers is triangle-major with
// fd2_stride(nq) pairs per triangle (a multiple of 16 bytes, so that a lane
// reads a triangle's values with 16-byte loads); the padding entry is unused.
constexpr int fd2_stride(int nq) { return (nq + 1) & ~1; }
// f2_ready: the workspace already holds the float-float density (written by
// the far sum's charge preparation), else it is converted first
void launch_apply_stream(const int64_t* row, const int32_t* ptri, const int32_t* ptgt, const float2* C2, int nq,
                         const double* f, int64_t N, int64_t P, int64_t M, double* u, void* ws, int32_t* flag,
                         int sm_count, cudaStream_t s, bool f2_ready = false);
