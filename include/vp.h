/*
 * vp.h - C ABI of libvp: the 2-D Poisson volume potential over a triangle
 * mesh on one NVIDIA GB300 (sm_103a), after Shen & Serkh, "Accelerating
 * potential evaluation over unstructured meshes in two dimensions"
 * (arXiv 2205.04401).
 *
 *     u(x) = int_Omega G(x, y) f(y) dA_y,     G(x, y) = (1/2pi) log|x - y|     (Section 1)
 *
 * evaluated by the subtract-and-add scheme of Section 3.6: a far sum over
 * every quadrature node as a point charge, corrected for the (target,
 * triangle) pairs whose near field (Section 4.1) or interior (Section 3.4)
 * holds the target.
 *
 * General conventions
 *  - Every function returns a vp_status (0 = VP_OK, negative = error) unless
 *    stated otherwise.  No function aborts, throws or exits; on error the
 *    output handles are left NULL and nothing is leaked.
 *  - "host" pointers are ordinary CPU memory and are read (or written) during
 *    the call only.  "device" pointers are CUDA global memory on the context's
 *    device, owned by the caller; they must stay valid until the given stream
 *    reaches the work that uses them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued asynchronously on it unless stated otherwise.
 *  - Handles (vp_ctx, vp_mesh, vp_nf) own their device memory until released.
 *    A vp_mesh / vp_nf must be released before the vp_ctx that made it.
 *  - Sizes are int64_t element counts; coordinates are interleaved (x, y)
 *    float64 pairs.
 */
#ifndef VP_H
#define VP_H

#include <stdint.h>

#if defined(__GNUC__)
#define VP_API __attribute__((visibility("default")))
#else
#define VP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vp_ctx vp_ctx;
typedef struct vp_mesh vp_mesh;
typedef struct vp_nf vp_nf;

typedef enum vp_status {
    VP_OK = 0,
    VP_ERR_INVALID_ARG = -1,     /* a NULL, negative or inconsistent argument */
    VP_ERR_DEGENERATE_TRI = -2,  /* a triangle with zero area (after CCW normalisation) */
    VP_ERR_NONFINITE = -3,       /* a NaN or Inf coordinate */
    VP_ERR_OOM = -4,             /* device allocation failed */
    VP_ERR_CUDA = -5,            /* any other CUDA runtime error (see vp_last_error) */
    VP_ERR_TIMEOUT = -6,         /* a bounded device wait ran out */
    VP_ERR_NO_DEVICE = -7,       /* no usable sm_103 device */
    VP_ERR_STATE = -8            /* handle used with the wrong context or after release */
} vp_status;

/* Far-field quadrature rules on the reference simplex (Section 3.2).  The two
 * built-in rules are S3-symmetric positive-interior rules derived from their
 * moment equations: 16 nodes exact to degree 8, 19 nodes exact to degree 9.
 * VP_RULE_CONICAL(n), n in [8, 50], is the conical-product Gauss rule of total
 * degree n for raising the far order (offloading, Section 4.2): with the
 * m = (n + 3)/2 (integer division) Gauss-Legendre points u_i and weights a_i
 * on [0, 1], node k = i m + j (i, j < m) is
 *   x_k = u_i,  y_k = (1 - u_i) u_j,  w_k = a_i a_j (1 - u_i),
 * m^2 nodes, positive weights, all inside the simplex, exact to degree
 * 2m - 2 >= n.  Its w-hat (Eq. rho0) is the largest weight among the
 * (n + 2)/2 nodes nearest an edge, maximised over the three edges, with the
 * nodes tied (to 1e-9 relative) with the last of them included.  The rule is
 * made on the host on first use in a context and kept until vp_destroy. */
typedef enum vp_rule { VP_RULE_16_D8 = 16, VP_RULE_19_D9 = 19 } vp_rule;
#define VP_RULE_CONICAL(n) (1000 + (n))
#define VP_RULE_CONICAL_MIN 8
#define VP_RULE_CONICAL_MAX 50
/* VP_RULE_SYM(n), n in {12, 20, 25, 30, 40, 50}: S3-symmetric rules of
 * degree n with positive weights and all nodes inside the simplex, about
 * two-thirds of the nodes of the conical rule of the same degree (33, 81,
 * 124, 175, 295 and 453 nodes; the Xiao-Gimbutas rules the paper takes have
 * 32 at degree 12, 290 at 40 and 444 at 50).  Each is the root of its S3-invariant moment
 * equations next to an orbit structure found by orbit elimination (a
 * symmetrised product rule reduced one orbit at a time, the equations
 * restored by Gauss-Newton after each step), computed in 90-digit
 * arithmetic and rounded once; nodes in orbit order (centroid, S21, S111).
 * w-hat as for the built-in rules. */
#define VP_RULE_SYM(n) (2000 + (n))

/* The nodes, weights, w-hat and degree of a far rule (host only, no device
 * needed).  x, y, w: host arrays of cap entries (each may be NULL); *n gets
 * the node count.  With cap < *n and any array non-NULL: INVALID_ARG.
 * Errors: INVALID_ARG (unknown rule). */
VP_API int vp_far_rule(int32_t rule, double* x, double* y, double* w, double* what, int32_t* degree, int32_t cap,
                       int32_t* n);

/* Arithmetic of vp_potential_eval.  VP_FP64: FP64 everywhere.  VP_MIXED: the
 * far sum in compensated FP32 (float-float coordinates and logarithm;
 * float-float partial sums over at most 2,048 sources, reduced in FP64); the
 * stored correction weights applied with
 * float-float products and FP64 sums (1 to 15 densities on the built-in far
 * rules) or in FP64 (16 or more densities, or a higher-order far rule).
 * VP_MIXED_TC: the far sum of VP_MIXED; the corrections applied on the tensor
 * cores from an exact split of C and f into L balanced base-128 digits held
 * as bf16 (vp_nf_prepare_tc), accumulated exactly in FP32 and combined in
 * FP64.  Its only error beyond VP_MIXED is the rounding of every weight to
 * 7L - 1 bits below the largest weight of its kind (near or self) for its
 * target, and of every density value to 7L - 1 bits below the largest value
 * of its density.  VP_MIXED_FMM: the corrections of VP_MIXED, the far sum by a
 * fast multipole method (the coupling of Section 3.6, where the paper calls a
 * library FMM): a uniform quadtree over the nodes and targets, complex
 * multipole and local expansions of 40 terms in FP64 with the Greengard-
 * Rokhlin translations, and the leaf and adjacent boxes summed directly in
 * float-float; its translations keep a point source at the nearest corner of
 * a well-separated box within 4e-16 of the direct value.  Its plan (tree,
 * sorted nodes and targets) is built on the first evaluation of a vp_nf,
 * which synchronises `stream`. */
typedef enum vp_precision { VP_FP64 = 0, VP_MIXED = 1, VP_MIXED_TC = 2, VP_MIXED_FMM = 3 } vp_precision;

/* Parameters of the near-field characterisation and correction weights. */
typedef struct vp_nf_params {
    double eps;        /* tolerance of Eq. (precise_far) for the un-normalised log kernel, |f| <= 1;
                          default 1e-12, accepted range [1e-15, 1e-2] */
    double c_far;      /* C_N of Eq. (rho0) for the far rule; 1 gives the provable superset E' */
    double c_near;     /* C_N for the degree-12 near rule (Table "C_N values": C_12 = 12) */
    int32_t depth_cap; /* maximum subdivision depth of Section 3.3; leaves at the cap are counted */
    int32_t flags;     /* 0, or VP_NF_FP64_WEIGHTS */
} vp_nf_params;

/* Fill *out with the defaults vp_nearfield_build uses when params is NULL:
 * eps 1e-12 (reading of the paper's experiments), c_far 1 (the provable
 * superset E' of Section 4.1), c_near 12 (Table "C_N values", C_12 = 12),
 * depth_cap 30, flags 0.  Host only; needs no device.  Errors: INVALID_ARG
 * (out NULL). */
VP_API int vp_nf_params_default(vp_nf_params* out);

/* vp_nf_params.flags: evaluate the node quadratures of the correction
 * weights in FP64.  By default they run in float-float arithmetic (pairs of
 * FP32 values with error-free transformations, ~2^-48 per operation), which
 * GB300 executes some 20x faster than FP64, and the self interaction's
 * radial sums take a 5-point rule that, like the 8-point generalized
 * Gaussian rule of the FP64 path (Section 3.4), is exact for the P_4
 * moments; the subdivision tree and every geometric predicate are FP64
 * (bit-exact) either way. */
#define VP_NF_FP64_WEIGHTS 1

/* Counters of Section 5 (c, s_n, s_l) and sizes of a near-field build. */
typedef struct vp_nf_stats_t {
    int64_t n_targets;      /* M */
    int64_t n_nodes;        /* N = n_tri * nq */
    int64_t n_pairs;        /* P = number of (target, triangle) corrections */
    int64_t n_self;         /* pairs with the target inside the triangle */
    int64_t n_near;         /* pairs with the target in the triangle's near field */
    int64_t near_leaves;    /* sum over near pairs of leaf sub-triangles (s_n * M) */
    int64_t self_panels;    /* sum over self pairs of arc-length panels (s_l * M) */
    int64_t depth_capped;   /* leaves stopped by depth_cap rather than the stop test */
    int64_t outside;        /* targets in no triangle */
    int64_t bytes_device;   /* device bytes held by the vp_nf */
    double build_ms;        /* wall time of vp_nearfield_build */
} vp_nf_stats_t;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (must be compute capability 10.3).
 * Allocates small constant tables, copies the log tables of the float-float
 * kernels and resolves the fixed scratch of vp_potential_eval_noalloc (so
 * that no later call loads a module or blocks on a table copy).  *out
 * receives the handle.  Errors: NO_DEVICE, OOM, CUDA. */
VP_API int vp_create(vp_ctx** out, int device);

/* Release the context.  NULL is ignored. */
VP_API void vp_destroy(vp_ctx* ctx);

/* Device memory held by the context itself: the evaluation workspace (grown
 * on demand by vp_potential_eval and kept for reuse) and the staging buffer
 * of vp_potential_eval_host.  Host only.  Errors: STATE. */
VP_API int vp_ctx_memory(const vp_ctx* ctx, int64_t* workspace_bytes, int64_t* staging_bytes);

/* Bound on the column scratch of the symmetric far sum (the node-target far
 * sum of VP_MIXED with one density, Section 3.6): the target tiles are
 * processed in bands whose column partial sums fit `bytes` (default 256 MiB;
 * accepted 1 MiB .. 1 TiB), so its workspace is about 1.25 x bytes + 40 N
 * bytes whatever the node count N.  Smaller caps mean more, shorter launches
 * and the same result up to the order of the FP64 additions.  Applies to
 * near fields whose first symmetric evaluation comes after the call.  Host
 * only.  Errors: STATE, INVALID_ARG. */
VP_API int vp_set_far_sym_cap(vp_ctx* ctx, int64_t bytes);

/* Human-readable name of a status code (static storage). */
VP_API const char* vp_status_str(int status);

/* Copy the last error message of this context into buf (always
 * NUL-terminated, truncated to len).  Returns VP_OK. */
VP_API int vp_last_error(const vp_ctx* ctx, char* buf, int32_t len);

/* ------------------------------------------------------------------ mesh */

/* Upload a straight-sided triangle mesh and build its quadrature nodes
 * (Theorem 3.1 with the affine map rho_T(xi, eta) = A + xi (B - A) + eta (C - A)):
 *   node j = T*nq + k at rho_T(xi_k, eta_k), weight W_j = w_k * J_T,
 *   J_T = (B - A) x (C - A) = 2 area(T) > 0.
 * vxy:  host, [nv][2] float64 vertex coordinates.
 * tri:  host, [nt][3] int32 vertex indices; clockwise triangles are made
 *       counter-clockwise by swapping their 2nd and 3rd vertex.
 * rule: VP_RULE_16_D8, VP_RULE_19_D9 or VP_RULE_CONICAL(n).  Meshes on a
 *       conical rule are evaluated with the FP64 correction apply in every
 *       precision, and VP_MIXED_TC, vp_nf_prepare_tc and the server refuse
 *       them (INVALID_ARG).
 * Errors: INVALID_ARG (index out of range, nt < 1, nt * nq > INT32_MAX),
 * NONFINITE, DEGENERATE_TRI.
 * The call synchronises `stream` before returning (it validates on device). */
VP_API int vp_mesh_upload(vp_ctx* ctx, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, int32_t rule,
                   void* stream, vp_mesh** out);

/* Same as vp_mesh_upload with DEVICE inputs: vxy_dev [nv][2] float64 and
 * tri_dev [nt][3] int32 in the context's device memory (validated on the
 * device: bad indices, non-finite or degenerate input give the same codes). */
VP_API int vp_mesh_upload_dev(vp_ctx* ctx, const double* vxy_dev, int64_t nv, const int32_t* tri_dev, int64_t nt,
                              int32_t rule, void* stream, vp_mesh** out);

/* Upload a mesh with curved elements (Section 3.1, blending map of Eq.
 * for:blend) from HOST arrays and build its nodes and weights (Theorem 3.1
 * with |det J_rho|).  A curved element is a counter-clockwise triangle
 * (v0, v1, v2) whose side v0 -> v1 is the curve c(xi), xi in [0, 1], given by
 * its deviation from the chord,
 *     c(xi) - (1 - xi) v0 - xi v1 = xi (1 - xi) D(xi),   D(xi) = sum_{k<=K} a_k T_k(2 xi - 1),
 * and mapped from the reference simplex by
 *     rho(xi, eta) = v0 + xi (v1 - v0) + eta (v2 - v0) + xi (1 - xi - eta) D(xi):
 *   node j = T*nq + k at rho_T(xi_k, eta_k), W_j = w_k det J_rho(xi_k, eta_k).
 * vxy, tri, rule: as vp_mesh_upload (straight triangles may be clockwise;
 *       curved ones must be counter-clockwise, else VP_ERR_INVALID_ARG).
 * cidx: host [nt] int32, the curve of each triangle, -1 for a straight one.
 * coef: host [ncurve][2][K+1] float64, the Chebyshev coefficients a_k of D,
 *       x then y (may be NULL when ncurve == 0); 0 <= K <= 64.
 * Near-field builds on such a mesh take, for a curved triangle: its chord
 * triangle for the near-field ellipses (the last remark of Section 4.1) and
 * J_T (the chord's 2 area) in the ellipse parameter; the curved element
 * itself for point location (the two straight sides' orientation tests and
 * the Newton preimage, eta >= 0) and for the correction weights (the
 * subdivision of Section 3.3 in reference coordinates mapped through rho;
 * the radius-arclength fans of Section 3.4 around rho^-1(x)).
 * Errors: those of vp_mesh_upload; INVALID_ARG for a curve index outside
 * [-1, ncurve) or K outside [0, 64]; NONFINITE for a non-finite coefficient;
 * DEGENERATE_TRI when det J_rho <= 0 at a node.  Synchronises `stream`. */
VP_API int vp_mesh_upload_curved(vp_ctx* ctx, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt,
                                 const int32_t* cidx, const double* coef, int64_t ncurve, int32_t K, int32_t rule,
                                 void* stream, vp_mesh** out);

/* Sizes of a mesh: triangles, nodes N = nt * nq, nodes per triangle nq. */
VP_API int vp_mesh_info(const vp_mesh* mesh, int64_t* n_tri, int64_t* n_nodes, int32_t* nq);

/* Copy node coordinates (device [N][2]) and node weights W (device [N]) into
 * caller buffers; either pointer may be NULL.  Density values are given at
 * these nodes, in this order (triangle-major: j = T*nq + k). */
VP_API int vp_mesh_nodes(const vp_mesh* mesh, double* yxy_dev, double* w_dev, void* stream);

/* Release a mesh.  NULL is ignored. */
VP_API void vp_mesh_release(vp_mesh* mesh);

/* ------------------------------------------------------------ near field */

/* Targets are the mesh nodes (if node_targets != 0), followed by m extra
 * points txy_dev (device [m][2] float64, may be NULL when m == 0).
 *
 * Builds, for every target x, the triangle S(x) containing it (Appendix A.5:
 * the lowest-index triangle whose three orientation tests are >= 0; a node's
 * own triangle for node targets) and N(x), the triangles T != S(x) whose
 * near field E_T holds x (Section 4.1, Eqs. rho0 / threeE): x lies in the open
 * Bernstein ellipse of some edge PQ of T with parameter
 *     rho0 = (w J_T / (eps C_N))^(1/N),
 * tested exactly as rho_x^N < w J_T / (eps C_N) with
 *     s = (|x-P| + |x-Q|) / |Q-P|,  rho_x = s + sqrt(max(s^2 - 1, 0)),
 * rho_x^N a left-to-right product, all in FP64 without fused multiply-add.
 * Then computes, per (x, T) pair, the nq correction weights
 *     C_k = w_k sum_a K_a(xi_k) m_a - [k != own(x)] W_k G(x, y_k),
 *     m_a = int_T G(x, y) K_a(rho_T^-1 y) dA,
 * with K_a the Koornwinder basis of P_4 (Section 2.1), by adaptive
 * subdivision (Section 3.3) for near pairs and radius-arclength fans
 * (Section 3.4) for self pairs.  The density on T is taken as its discrete
 * L2 projection onto P_4 with the far rule.
 * params may be NULL (defaults: eps 1e-12, c_far 1, c_near 12, depth_cap 30).
 * The call synchronises `stream`.  Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
VP_API int vp_nearfield_build(vp_ctx* ctx, const vp_mesh* mesh, int32_t node_targets, const double* txy_dev, int64_t m,
                       const vp_nf_params* params, void* stream, vp_nf** out);

/* Same as vp_nearfield_build with the extra targets in a HOST buffer
 * (txy_host [m][2], may be NULL when m = 0): copied to the device through the
 * context's staging buffer on `stream`, then built.  Synchronises `stream`. */
VP_API int vp_nearfield_build_host(vp_ctx* ctx, const vp_mesh* mesh, int32_t node_targets, const double* txy_host,
                                   int64_t m, const vp_nf_params* params, void* stream, vp_nf** out);

/* Counters and sizes of a build (host struct). */
VP_API int vp_nf_stats(const vp_nf* nf, vp_nf_stats_t* out);

/* Copy the target-major lists into caller device buffers (any may be NULL):
 * row_ptr [M+1] int64, tri [P] int32 ascending within a row, kind [P] uint8
 * (1 = self, 0 = near), tself [M] int32 (S(x), -1 outside). */
VP_API int vp_nf_lists(const vp_nf* nf, int64_t* row_ptr_dev, int32_t* tri_dev, uint8_t* kind_dev, int32_t* tself_dev,
                void* stream);

/* Copy the correction weights, device [P][nq] float64, row order of vp_nf_lists. */
VP_API int vp_nf_weights(const vp_nf* nf, double* w_dev, void* stream);

/* Release a near-field build.  NULL is ignored. */
VP_API void vp_nf_release(vp_nf* nf);

/* Plan of the tensor-core correction apply (VP_MIXED_TC; the last sum of the
 * subtract-and-add evaluation, Section 3.6, as a block-sparse times dense
 * product).  Targets are ordered along a Morton curve and cut into tiles of
 * 128; each tile's near-field rows become one dense block row over the union
 * of its triangles (24 columns per triangle; near and self pairs in separate
 * runs with their own row exponents), its weights split into `levels`
 * (3, 4 or 5) bf16 digit planes and stored on the device, levels x 2 bytes
 * per entry of the dense rows (see vp_nf_tc_info).  The weights and densities
 * are rounded to 7 levels - 1 bits below their run/density maximum: 5 levels
 * hold the synthetic star workloads within 1e-10 of the FP64 result, 4 and
 * 3 levels within about 3e-9 and 5e-7.
 * Replaces an earlier plan of nf; synchronises `stream`.
 * Errors: VP_ERR_INVALID_ARG for other levels or when a tile holds more than
 * 16384 near pairs (then use VP_MIXED); VP_ERR_OOM; VP_ERR_CUDA. */
VP_API int vp_nf_prepare_tc(vp_ctx* ctx, vp_nf* nf, int32_t levels, void* stream);

/* Synchronise `stream`, then report and clear the device-side error flags of
 * the context's asynchronous kernels (VP_ERR_TIMEOUT when a bounded wait of
 * the tensor-core apply gave up; its output is then not valid). */
VP_API int vp_device_status(vp_ctx* ctx, void* stream);

/* The tensor-core plan of nf: digits, tiles, chunks of 48 columns and
 * device bytes (all 0 without a plan).  Any pointer may be NULL. */
VP_API int vp_nf_tc_info(const vp_nf* nf, int32_t* levels, int64_t* n_tiles, int64_t* n_chunks, int64_t* bytes);

/* The fast-multipole plan of nf (VP_MIXED_FMM): leaf level of its quadtree
 * (chosen per build from a cost model of direct pairs against translations)
 * and the number of boxes over all levels; 0 before the first VP_MIXED_FMM
 * evaluation.  Either pointer may be NULL. */
VP_API int vp_nf_fmm_info(const vp_nf* nf, int32_t* leaf_level, int64_t* n_boxes);

/* ------------------------------------------------------------- evaluation */

/* u = far + corrections (Section 3.6) for d densities.
 * f_dev: device [d][N] float64 density values at the mesh nodes.
 * u_dev: device [d][M] float64 output, fully overwritten.
 * precision: VP_FP64, VP_MIXED or VP_MIXED_TC.  1 <= d <= 256.  VP_MIXED_TC
 * builds the tensor-core plan with 5 digits on first use if
 * vp_nf_prepare_tc was not called (that first call synchronises `stream`).
 * Uses workspace owned by the context: calls on one context must be issued
 * on one stream (or serialised by the caller). */
VP_API int vp_potential_eval(vp_ctx* ctx, const vp_nf* nf, const double* f_dev, int32_t d, double* u_dev,
                      int32_t precision, void* stream);

/* Same as vp_potential_eval with HOST buffers (f_host [d][N], u_host [d][M]):
 * copies in, evaluates, copies out and synchronises `stream` before return. */
VP_API int vp_potential_eval_host(vp_ctx* ctx, const vp_nf* nf, const double* f_host, int32_t d, double* u_host,
                           int32_t precision, void* stream);

/* Same computation and arguments as vp_potential_eval, but it allocates no
 * device memory, for callers that cannot: a process whose GPU memory is
 * owned by another allocator (a caching allocator can hold every free byte,
 * so cudaMalloc fails), or a serving loop that cannot accept the device-wide
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart.
 * Its scratch (split-source partial sums and float-float charges) lives in a
 * fixed 32 MiB device array compiled into the library, which every GPU that
 * loads the library holds until the process exits.  A call that would need
 * more (about splits * d * M * 8 + N * 2 * min(d, 8) * 4 bytes) is rejected
 * with VP_ERR_INVALID_ARG and a message; use vp_potential_eval then.
 * vp_create has already resolved the array's device address
 * (cudaGetSymbolAddress, which loads the module that holds it) and copied the
 * float-float log tables, so this call allocates nothing, copies no table and
 * looks up no symbol, on its first call as on every later one.
 * All calls share the one array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other contexts on the
 * same device) race on it and must be serialised by the caller.  Nothing in
 * it needs to start at zero. */
VP_API int vp_potential_eval_noalloc(vp_ctx* ctx, const vp_nf* nf, const double* f_dev, int32_t d, double* u_dev,
                                     int32_t precision, void* stream);

/* One evaluation of a batch: a near-field build with its densities/output. */
typedef struct vp_eval_item {
    const vp_nf* nf;
    const double* f_dev;   /* device [d][N] */
    int32_t d;
    double* u_dev;         /* device [d][M] */
} vp_eval_item;

/* A prepared batch of evaluations over many near-field builds (possibly
 * different meshes and density counts).  vp_batch_create validates the items,
 * builds the work list of a persistent far-sum kernel (work units: an item's
 * block of target rows, taken from an atomic counter so uneven meshes
 * balance; one launch per density-chunk width 1/2/4/8) and of one correction
 * launch over all items' targets, picks the targets-per-thread tile of the
 * far sum by timing the variants once per context (autotuning, on the
 * first batch), and captures the whole launch sequence in a CUDA graph.
 * The item pointers (f_dev, u_dev) are read at every launch, so new
 * densities can be written in place and the batch relaunched.
 * vp_batch_launch replays the graph on `stream` (asynchronous).  Results
 * agree with vp_potential_eval item by item up to the order of the far-sum
 * partial sums.  The batch holds device descriptors and charge buffers
 * (about N * 2 * min(d, 8) floats per item) until released.
 * precision: VP_FP64, VP_MIXED, or VP_MIXED_FMM (then the graph holds every
 * item's multipole evaluation in turn, with one workspace for the largest
 * item; the items' multipole plans are built by vp_batch_create). */
typedef struct vp_batch vp_batch;
VP_API int vp_batch_create(vp_ctx* ctx, const vp_eval_item* items, int32_t n, int32_t precision, void* stream,
                           vp_batch** out);
VP_API int vp_batch_launch(vp_batch* batch, void* stream);
VP_API void vp_batch_release(vp_batch* batch);

/* Tile of the batched far sum for density-chunk width `width` (1, 2, 4 or 8):
 * targets_per_thread 1, 2 or 4 fixes it for batches created afterwards on
 * this context; 0 (the default) lets vp_batch_create's autotuner choose.
 * Every tile sums each target's sources in the same order, so the results do
 * not depend on it.  Host only.  Errors: STATE, INVALID_ARG. */
VP_API int vp_set_batch_tile(vp_ctx* ctx, int32_t width, int32_t targets_per_thread);

/* The tile and the work-unit count of each density-chunk width of a batch
 * (index 0..3 for widths 1, 2, 4, 8; 0 where the batch has no such chunk or
 * runs the multipole path).  Either pointer may be NULL.  Errors: STATE. */
VP_API int vp_batch_info(const vp_batch* batch, int32_t* targets_per_thread, int64_t* work_units);

/* Evaluate n items at once: vp_batch_create + vp_batch_launch + release
 * (synchronises `stream`). */
VP_API int vp_potential_eval_batch(vp_ctx* ctx, const vp_eval_item* items, int32_t n, int32_t precision, void* stream);

/* --------------------------------------------------------------- serving */

/* A serving loop with continuous batching (no counterpart in the paper; it
 * serves the evaluation of Section 3.6 to a stream of requests).  A worker
 * thread owns `slots` CUDA streams.  Requests wait in a FIFO queue and are
 * admitted as soon as a slot is free and their device footprint (densities
 * d*N*8 B, output d*M*8 B, evaluation workspace) fits in hbm_budget_bytes
 * next to the requests already running; each runs H2D copy, the evaluation
 * of vp_potential_eval and the D2H copy on its slot's stream, so requests
 * that arrive while others run overlap with them on the device.  A result
 * does not depend on what else is in flight.  Registered near-field builds
 * stay resident; "cold" meshes (host arrays) are uploaded and built (targets
 * = nodes, default parameters) on their first request, whose latency
 * includes the build.  Requests larger than the budget fail with
 * VP_ERR_OOM.  While a server runs, the context must not be used from other
 * threads except through the server (it shares the context's tables). */
typedef struct vp_server vp_server;

typedef struct vp_server_stats_t {
    int64_t completed, failed, queued, cold_builds;
    int64_t evals;            /* sum over completed requests of d * M */
    int64_t peak_bytes;       /* largest admitted device footprint */
    int32_t max_concurrent;   /* most requests running at once */
    int32_t reserved;
    double p50_ms, p99_ms;    /* latency from submission to result */
    double p50_wait_ms;       /* time from submission to admission */
    double evals_per_s;       /* evals / (last completion - first submission) */
} vp_server_stats_t;

/* precision: VP_FP64, VP_MIXED or VP_MIXED_FMM (the multipole plan of a mesh
 * is built when it is registered, or right after a cold mesh's build). */
VP_API int vp_server_create(vp_ctx* ctx, int32_t slots, int64_t hbm_budget_bytes, int32_t precision,
                            vp_server** out);
/* Serve requests against an existing near-field build (the caller keeps it
 * alive until vp_server_destroy). */
VP_API int vp_server_register(vp_server* server, int64_t key, const vp_nf* nf);
/* Register host mesh arrays (copied) to be built on the first request. */
VP_API int vp_server_register_cold(vp_server* server, int64_t key, const double* vxy, int64_t nv, const int32_t* tri,
                                   int64_t nt, int32_t rule);
/* N (nodes) and M (targets) of a registered mesh (cold: M = N). */
VP_API int vp_server_mesh_size(vp_server* server, int64_t key, int64_t* n_nodes, int64_t* n_targets);
/* Queue one request: f_host [d][N] densities, u_host [d][M] result, both host
 * memory that must stay valid until the request completes (page-locked
 * memory lets the copies overlap; pageable memory works but serialises the
 * scheduler on each copy).  *ticket identifies the request. */
VP_API int vp_server_submit(vp_server* server, int64_t key, const double* f_host, int32_t d, double* u_host,
                            int64_t* ticket);
/* Block until the request completes (VP_ERR_TIMEOUT after timeout_s);
 * *status is the request's own status, *latency_ms its submission-to-result
 * time. */
VP_API int vp_server_wait(vp_server* server, int64_t ticket, double timeout_s, int32_t* status, double* latency_ms);
VP_API int vp_server_stats(vp_server* server, vp_server_stats_t* out);
/* Drain the queue, stop the worker and release the server's streams and
 * cold builds. */
VP_API void vp_server_destroy(vp_server* server);

/* ------------------------------------------------------------- profiling */

/* Per-stage GPU timing.  When enabled, the library records a CUDA event pair
 * on the caller's stream around each kernel stage; vp_profile_read returns,
 * for every stage, its name, the number of launches timed and their summed
 * device time in milliseconds (it synchronises the device first).
 * vp_profile_reset clears the accumulators.  Off by default. */
VP_API int vp_profile_enable(vp_ctx* ctx, int32_t on);
VP_API int vp_profile_reset(vp_ctx* ctx);
/* names: caller buffer of cap * 32 chars (NUL-padded); counts, ms: [cap].
 * *n receives the number of stages (at most cap are written). */
VP_API int vp_profile_read(vp_ctx* ctx, char* names, int64_t* counts, double* ms, int32_t cap, int32_t* n);

/* --------------------------------------------------------- interpolation */

/* Interpolation of the potential over the elements of an interpolation mesh
 * (Section 3.5), e.g. a mesh staggered with the quadrature mesh (Section
 * 4.3), so that u can be evaluated anywhere from one evaluation at the
 * interpolation nodes.  On each element Delta with map rho (affine, or the
 * blending map of a curved element) the Koornwinder expansion of u o rho of
 * degree N_s (`order`, 1..20) comes from u at dim P_{N_s} = (N_s+1)(N_s+2)/2
 * interpolation nodes by the inverse interpolation matrix, and
 * u(x) = I(rho^{-1}(x)) (the affine inverse, or Newton's method on curved
 * elements).  The nodes are the Blyth-Pozrikidis construction on the N_s+1
 * Gauss-Legendre points (all inside the element, S3-symmetric; the paper's
 * Vioreanu-Rokhlin tables are not used), node (i, j, k), i + j + k = N_s, at
 *     xi = (1 + 2 v_i - v_j - v_k)/3, eta = (1 + 2 v_j - v_i - v_k)/3,
 * v the Gauss-Legendre points mapped to [0, 1], ordered by j, then i.
 * vxy, tri: host arrays as vp_mesh_upload; cidx, coef, ncurve, K: curved
 * elements as vp_mesh_upload_curved, or cidx = NULL for a straight mesh.
 * Errors: those of the mesh uploads; INVALID_ARG for order outside 1..20. */
typedef struct vp_interp vp_interp;
VP_API int vp_interp_create(vp_ctx* ctx, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt,
                            const int32_t* cidx, const double* coef, int64_t ncurve, int32_t K, int32_t order,
                            void* stream, vp_interp** out);
/* Elements, nodes (n_tri * nodes_per_tri) and nodes per element. */
VP_API int vp_interp_info(const vp_interp* interp, int64_t* n_tri, int64_t* n_nodes, int32_t* nodes_per_tri);
/* Node coordinates, device [n_nodes][2], element-major: the targets at which
 * the potential is evaluated (extra targets of vp_nearfield_build). */
VP_API int vp_interp_nodes(const vp_interp* interp, double* xy_dev, void* stream);
/* Expansion coefficients: u_dev device [d][n_nodes] values at the nodes ->
 * coef_dev device [d][n_tri][nodes_per_tri] (Koornwinder index
 * n (n + 1)/2 + m of K_mn, Section 2.1). */
VP_API int vp_interp_coeffs(vp_interp* interp, const double* u_dev, int32_t d, double* coef_dev, void* stream);
/* u at m points pts_dev (device [m][2]) -> out_dev device [d][m]; elem_dev
 * (device [m] int32, may be NULL) receives the element of each point (the
 * lowest-index element that holds it, Appendix A.5); points in no element
 * give NaN and -1. */
VP_API int vp_interp_eval(vp_interp* interp, const double* coef_dev, int32_t d, const double* pts_dev, int64_t m,
                          double* out_dev, int32_t* elem_dev, void* stream);
VP_API void vp_interp_release(vp_interp* interp);

/* ---------------------------------------------------------------- tables */

/* The compiled quadrature tables, for inspection (host buffers of capacity
 * cap; *n receives the node count).  which: 16 / 19 (far rules), 33 (near
 * rule: the S3-symmetric rule of degree 12), 8 (radial generalized Gaussian rule: x = r, y unused), 5 (the
 * radial rule of the float-float self weights: x = r, w = weights of int_0^1 r p(r) dr, y = weights of
 * int_0^1 r log(r) p(r) dr, both exact for deg p <= 4), 116 (the
 * arc-length Gauss-Legendre rule on [0,1]).  *what receives w of Eq. rho0
 * (0 for the 1-D rules). */
VP_API int vp_rule_table(int32_t which, double* x, double* y, double* w, double* what, int32_t cap, int32_t* n);

#ifdef __cplusplus
}
#endif

#endif /* VP_H */
