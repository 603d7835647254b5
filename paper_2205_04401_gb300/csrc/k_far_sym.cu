// Symmetric float-float far sum for the node targets (Section 3.6: all
// nodes act as charges q_j = W_j f_j; with the nodes as targets, G(x_i, y_j) =
// G(x_j, y_i)).  Every unordered pair of nodes in different target tiles has
// its float-float distance and logarithm evaluated once and used twice:
//
//   row:    u_i += q_j G_ij      (target i of tile I, source j beyond tile I)
//   column: u_j += q_i G_ij
//
// Work units are (tile I of 512 nodes, 2048 consecutive nodes beyond it).
// The tiles are cut into bands of consecutive tiles whose column ranges hold
// at most a fixed number of values (vp_set_far_sym_cap, 256 MiB by default),
// so the scratch is bounded whatever N: per band, one launch writes the row
// sums of its units to rowbuf[unit] and the column sums to colbuf[I][j], and
// an accumulation pass adds, node by node in a fixed order, the rows of the
// node's own tile and the columns of the band's tiles before it into an FP64
// accumulator.  Equal column capacity per band means equal work per band
// (pairs = 512 x column values).  The pairs inside a tile take the one-sided
// kernel (own node excluded); a last pass adds that diagonal part.  Every
// write has one owner, so the result does not depend on scheduling.
//
// Inside a unit a warp sweeps 32 sources against its 32 lanes x 4 targets in
// 32 rotation steps (lane l takes source (l + k) mod 32 at step k), so each
// source's column sum is updated by one lane at a time in the warp's own
// shared-memory accumulator; the four warps' accumulators are added at the
// end of every 128-source tile in float-float.  The distance, logarithm and
// per-pair accumulation arithmetic is that of the one-sided kernel
// (vp_ff.cuh); a row sum stays float-float over its unit's 2,048 sources and
// is converted to FP64 once.
#include <algorithm>
#include <vector>

#include "vp_internal.h"
#include "vp_ff.cuh"

namespace {

constexpr int SYM_THREADS = 128;
constexpr int SYM_TPT = 4;
constexpr int SYM_TI = SYM_THREADS * SYM_TPT;   // target tile
constexpr int SYM_TJ = 128;                     // source tile in shared memory
constexpr int SYM_UJ = 16;                      // source tiles per work unit

struct SymSmem {
    float4 sxy[SYM_TJ];
    float2 sq[SYM_TJ];                 // charge (h, l)
    float2 col[SYM_THREADS / 32][SYM_TJ];   // per-warp column accumulators (h, l)
    float4 stab[LOG_N];
};

__device__ __forceinline__ void two_sum_s(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Block b takes unit u = u0 + b of the band; unit -> (tile I, sources [j0, j1)).
// rowbuf[(u - u0) 512 + r], colbuf[coff[I] - cb0 + (j - (I + 1) 512)].
__global__ void __launch_bounds__(SYM_THREADS) k_far_sym(const float* __restrict__ shi, const float* __restrict__ slo,
                                                         const float* __restrict__ q, int64_t N,
                                                         const int32_t* __restrict__ unit_I,
                                                         const int64_t* __restrict__ unit_j0,
                                                         const int64_t* __restrict__ unit_j1,
                                                         const int64_t* __restrict__ coff, int64_t u0, int64_t cb0,
                                                         double* __restrict__ rowbuf, double* __restrict__ colbuf) {
    __shared__ SymSmem sm;
    for (int i = threadIdx.x; i < LOG_N; i += SYM_THREADS) sm.stab[i] = g_logtab_far.e[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t u = u0 + blockIdx.x;
    const int I = unit_I[u];
    const int64_t j0 = unit_j0[u], j1 = unit_j1[u];
    const int64_t jstart = (int64_t)(I + 1) * SYM_TI;
    float thx[SYM_TPT], thy[SYM_TPT], tlx[SYM_TPT], tly[SYM_TPT], qh[SYM_TPT], ql[SYM_TPT];
    bool active[SYM_TPT];
#pragma unroll
    for (int r = 0; r < SYM_TPT; r++) {
        const int64_t t = (int64_t)I * SYM_TI + r * SYM_THREADS + threadIdx.x;
        active[r] = t < N;
        thx[r] = active[r] ? shi[2 * t] : 0.f;
        thy[r] = active[r] ? shi[2 * t + 1] : 0.f;
        tlx[r] = active[r] ? slo[2 * t] : 0.f;
        tly[r] = active[r] ? slo[2 * t + 1] : 0.f;
        qh[r] = active[r] ? q[2 * t] : 0.f;             // inactive targets carry no charge
        ql[r] = active[r] ? q[2 * t + 1] : 0.f;
    }
    // row sums in float-float across the unit, renormalised after every
    // source tile (the FP64 pipe, 1/64 of the FP32 rate here, only converts
    // the unit's result)
    float sh[SYM_TPT], sl[SYM_TPT];
#pragma unroll
    for (int r = 0; r < SYM_TPT; r++) sh[r] = sl[r] = 0.f;
    for (int64_t base = j0; base < j1; base += SYM_TJ) {
        const int nt = (int)min((int64_t)SYM_TJ, j1 - base);
        __syncthreads();
        for (int i = threadIdx.x; i < SYM_TJ; i += SYM_THREADS) {
            if (i < nt) {
                const int64_t j = base + i;
                sm.sxy[i] = make_float4(shi[2 * j], shi[2 * j + 1], slo[2 * j], slo[2 * j + 1]);
                sm.sq[i] = make_float2(q[2 * j], q[2 * j + 1]);
            }
#pragma unroll
            for (int ww = 0; ww < SYM_THREADS / 32; ww++) sm.col[ww][i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2* col = sm.col[w];
        for (int sb = 0; sb < nt; sb += 32) {
#pragma unroll 2
            for (int k = 0; k < 32; k++) {
                const int jl = sb + ((lane + k) & 31);
                if (jl < nt) {
                    const float4 sv = sm.sxy[jl];
                    const float2 qj = sm.sq[jl];
                    float ch = 0.f, cl = 0.f;                      // column contribution of this lane
#pragma unroll
                    for (int r = 0; r < SYM_TPT; r++) {
                        float s, corr, lh, ll;
                        ff_dist2_far<false>(thx[r], thy[r], tlx[r], tly[r], sv, s, corr);   // distinct nodes
                        ff_log_far(sm.stab, s, corr, lh, ll);     // log |x_i - y_j|^2
                        ff_madd(qj.x, qj.y, lh, ll, sh[r], sl[r]);
                        if (r == 0) {                              // the column sum starts at this product
                            ch = __fmul_rn(qh[0], lh);
                            cl = __fmaf_rn(qh[0], ll, __fmaf_rn(ql[0], lh, __fmaf_rn(qh[0], lh, -ch)));
                        } else {
                            ff_madd(qh[r], ql[r], lh, ll, ch, cl);
                        }
                    }
                    const float2 c = col[jl];
                    float cs, ce;
                    two_sum_s(c.x, ch, cs, ce);
                    col[jl] = make_float2(cs, __fadd_rn(c.y, __fadd_rn(ce, cl)));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < SYM_TPT; r++) {                        // |sl| back to half an ulp of sh
            float h, e;
            two_sum_s(sh[r], sl[r], h, e);
            sh[r] = h;
            sl[r] = e;
        }
        __syncthreads();
        // column sums of this tile: the four warps' accumulators added in
        // float-float in a fixed order, then one conversion
        for (int i = threadIdx.x; i < nt; i += SYM_THREADS) {
            float2 c = sm.col[0][i];
#pragma unroll
            for (int ww = 1; ww < SYM_THREADS / 32; ww++) {
                const float2 d = sm.col[ww][i];
                float h, e;
                two_sum_s(c.x, d.x, h, e);
                c = make_float2(h, __fadd_rn(c.y, __fadd_rn(e, d.y)));
            }
            colbuf[coff[I] - cb0 + (base + i - jstart)] = (double)c.x + (double)c.y;
        }
    }
#pragma unroll
    for (int r = 0; r < SYM_TPT; r++)
        if (active[r]) rowbuf[(u - u0) * SYM_TI + r * SYM_THREADS + threadIdx.x] = (double)sh[r] + (double)sl[r];
}

// Pairs inside each tile, one-sided with the own node excluded: block I.
__global__ void __launch_bounds__(FF_THREADS) k_far_sym_diag(const float* __restrict__ shi, const float* __restrict__ slo,
                                                             const float* __restrict__ q, int64_t N,
                                                             const int32_t* __restrict__ tnode, double* __restrict__ diag) {
    __shared__ FFSmem<1> sm;
    ff_load_table(sm);
    const int64_t j0 = (int64_t)blockIdx.x * SYM_TI, j1 = min(N, j0 + SYM_TI);
    ff_far_block<1, SYM_TPT>(sm, shi, slo, q, j0, j1, shi, slo, tnode, N, j0 + threadIdx.x, 1, 0, diag);
}

// One band (tiles [tile0, tile1), units from u0, columns from cb0): for every
// node i >= tile0 512, s = the row sums of i's tile if it is in the band (its
// units in order) + the band's column sums of tiles I' < tile(i) (ascending);
// acc[i] = s on the first band, acc[i] += s after.
__global__ void k_far_sym_accum(const double* __restrict__ rowbuf, const double* __restrict__ colbuf,
                                const int64_t* __restrict__ ufirst, const int64_t* __restrict__ coff, int64_t N,
                                int tile0, int tile1, int64_t u0, int64_t cb0, int first, double* __restrict__ acc) {
    const int64_t i = (int64_t)tile0 * SYM_TI + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int I = (int)(i / SYM_TI);
    double s = 0.0;
    if (I < tile1) {
        const int64_t loc = i - (int64_t)I * SYM_TI;
        for (int64_t u = ufirst[I]; u < ufirst[I + 1]; u++) s += rowbuf[(u - u0) * SYM_TI + loc];
    }
    const int Iend = min(I, tile1);
    for (int Ip = tile0; Ip < Iend; Ip++) s += colbuf[coff[Ip] - cb0 + (i - (int64_t)(Ip + 1) * SYM_TI)];
    acc[i] = first ? s : acc[i] + s;
}

// u[i] = diag[i] + acc[i] / 4pi (acc sums log r^2)
__global__ void k_far_sym_combine(const double* __restrict__ diag, const double* __restrict__ acc, int64_t N,
                                  double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[i] = diag[i] + acc[i] * (0.5 * VP_INV_TWO_PI);
}

// Targets that are not nodes (t in [N, M)): one-sided, sources split over
// blockIdx.y; partial[split][t - N].
__global__ void __launch_bounds__(FF_THREADS) k_far_extra(const float* __restrict__ shi, const float* __restrict__ slo,
                                                          const float* __restrict__ q, int64_t N,
                                                          const float* __restrict__ thi, const float* __restrict__ tlo,
                                                          const int32_t* __restrict__ tnode, int64_t M, int splits,
                                                          double* __restrict__ partial) {
    __shared__ FFSmem<1> sm;
    ff_load_table(sm);
    const int split = blockIdx.y;
    const int64_t per = (N + splits - 1) / splits;
    const int64_t j0 = split * per, j1 = min(N, j0 + per);
    const int64_t m = M - N;
    const int64_t tbase = (int64_t)blockIdx.x * (FF_THREADS * SYM_TPT) + threadIdx.x;
    // the extra targets as a target set of their own: t' = t - N
    ff_far_block<1, SYM_TPT>(sm, shi, slo, q, j0, j1, thi + 2 * N, tlo + 2 * N, tnode + N, m, tbase, 1, 0,
                             partial + (int64_t)split * m);
}

__global__ void k_far_extra_reduce(const double* __restrict__ partial, int splits, int64_t n, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    for (int k = 0; k < splits; k++) v += partial[(int64_t)k * n + i];
    out[i] = v;
}

}  // namespace

// ---------------------------------------------------------------- host
bool far_sym_applicable(const vp_nf* nf, int d) {
    return d == 1 && nf->node_targets && nf->mesh->N >= 16 * SYM_TI;
}

// A band of consecutive target tiles [tile0, tile1) with its units
// [u0, u1) and its column values [c0, c1) (offsets into the global column
// layout coff).
struct SymBand {
    int tile0 = 0, tile1 = 0;
    int64_t u0 = 0, u1 = 0, c0 = 0, c1 = 0;
};

// Unit tables, kept with the near field (they depend on N and the cap only).
struct SymPlan {
    int64_t N = 0, n_units = 0, n_tiles = 0, col_len = 0;
    int64_t max_band_units = 0, max_band_cols = 0;
    std::vector<SymBand> bands;
    int32_t* unit_I = nullptr;
    int64_t *unit_j0 = nullptr, *unit_j1 = nullptr, *ufirst = nullptr, *coff = nullptr;
};

void far_sym_plan_free(SymPlan* p) {
    if (!p) return;
    cudaFree(p->unit_I);
    cudaFree(p->unit_j0);
    cudaFree(p->unit_j1);
    cudaFree(p->ufirst);
    cudaFree(p->coff);
    delete p;
}

static int64_t sym_units(int64_t N, std::vector<int32_t>* uI, std::vector<int64_t>* u0, std::vector<int64_t>* u1,
                         std::vector<int64_t>* uf, std::vector<int64_t>* co, int64_t* col_len,
                         std::vector<SymBand>* bands, int64_t cap) {
    const int64_t nI = (N + SYM_TI - 1) / SYM_TI;
    int64_t units = 0, cl = 0;
    SymBand cur;
    for (int64_t I = 0; I < nI; I++) {
        if (uf) uf->push_back(units);
        if (co) co->push_back(cl);
        const int64_t js = (I + 1) * SYM_TI;
        const int64_t len = js < N ? N - js : 0;
        // close the current band if this tile's columns would overflow it
        if (cur.tile1 > cur.tile0 && cur.c1 - cur.c0 + len > cap) {
            if (bands) bands->push_back(cur);
            cur = SymBand();
            cur.tile0 = cur.tile1 = (int)I;
            cur.u0 = cur.u1 = units;
            cur.c0 = cur.c1 = cl;
        }
        cur.tile1 = (int)I + 1;
        if (len > 0) {
            cl += len;
            for (int64_t j = js; j < N; j += (int64_t)SYM_TJ * SYM_UJ) {
                if (uI) {
                    uI->push_back((int32_t)I);
                    u0->push_back(j);
                    u1->push_back(std::min(N, j + (int64_t)SYM_TJ * SYM_UJ));
                }
                units++;
            }
        }
        cur.u1 = units;
        cur.c1 = cl;
    }
    if (bands && cur.tile1 > cur.tile0) bands->push_back(cur);
    if (uf) uf->push_back(units);
    if (co) co->push_back(cl);
    *col_len = cl;
    return units;
}

// Column values per band: the context's cap (vp_set_far_sym_cap) in FP64 values.
static int64_t sym_cap_values(const vp_ctx* ctx) { return std::max<int64_t>(ctx->far_sym_cap_bytes / 8, 1); }

static void band_maxima(const std::vector<SymBand>& bands, int64_t* mu, int64_t* mc) {
    *mu = *mc = 0;
    for (const SymBand& b : bands) {
        *mu = std::max(*mu, b.u1 - b.u0);
        *mc = std::max(*mc, b.c1 - b.c0);
    }
}

// Source splits of the extra-target sum: about 16 blocks per SM (more than two
// waves of the resident blocks), so that few targets still fill the GPU and
// the last wave is short (4 per SM left half the block slots empty).
static int extra_splits(int64_t N, int64_t m, int sm_count) {
    if (m <= 0) return 0;
    const int64_t blocks = (m + SYM_TI - 1) / SYM_TI;
    int64_t sp = (16LL * sm_count + blocks - 1) / blocks;
    sp = std::min<int64_t>(sp, std::max<int64_t>(1, N / 1024));
    return (int)std::max<int64_t>(1, std::min<int64_t>(sp, 256));
}

// [rowbuf: largest band's units x 512][colbuf: largest band's columns][acc N]
// [diag N][charges N x 2 floats][extra-target partials]
// (the plan's own band sizes once it exists, else those the context's cap gives)
size_t far_sym_ws_bytes(const vp_ctx* ctx, const vp_nf* nf) {
    const int64_t N = nf->mesh->N, m = nf->M - N;
    int64_t cl = 0, mu = 0, mc = 0;
    if (nf->sym) {
        mu = nf->sym->max_band_units;
        mc = nf->sym->max_band_cols;
    } else {
        std::vector<SymBand> bands;
        sym_units(N, nullptr, nullptr, nullptr, nullptr, nullptr, &cl, &bands, sym_cap_values(ctx));
        band_maxima(bands, &mu, &mc);
    }
    const int sp = extra_splits(N, m, ctx->sm_count);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al((size_t)mu * SYM_TI * 8) + al((size_t)mc * 8) + 2 * al((size_t)N * 8) +
           al((size_t)N * 2 * sizeof(float)) + al((size_t)sp * std::max<int64_t>(m, 0) * 8) + 256;
}

int far_sym_plan(vp_ctx* ctx, vp_nf* nf) {
    if (nf->sym) return VP_OK;
    const int64_t N = nf->mesh->N;
    std::vector<int32_t> uI;
    std::vector<int64_t> u0, u1, uf, co;
    SymPlan* p = new SymPlan();
    p->N = N;
    p->n_tiles = (N + SYM_TI - 1) / SYM_TI;
    p->n_units = sym_units(N, &uI, &u0, &u1, &uf, &co, &p->col_len, &p->bands, sym_cap_values(ctx));
    band_maxima(p->bands, &p->max_band_units, &p->max_band_cols);
    const size_t nu = std::max<int64_t>(p->n_units, 1);
    bool ok = cudaMalloc(&p->unit_I, nu * 4) == cudaSuccess && cudaMalloc(&p->unit_j0, nu * 8) == cudaSuccess &&
              cudaMalloc(&p->unit_j1, nu * 8) == cudaSuccess &&
              cudaMalloc(&p->ufirst, uf.size() * 8) == cudaSuccess && cudaMalloc(&p->coff, co.size() * 8) == cudaSuccess;
    if (ok && p->n_units) {
        ok = cudaMemcpy(p->unit_I, uI.data(), uI.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(p->unit_j0, u0.data(), u0.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(p->unit_j1, u1.data(), u1.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (ok)
        ok = cudaMemcpy(p->ufirst, uf.data(), uf.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(p->coff, co.data(), co.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        far_sym_plan_free(p);
        return vp_set_error(ctx, VP_ERR_OOM, "symmetric far-sum plan: allocation failed");
    }
    nf->sym = p;
    return VP_OK;
}

// u_far for one density: the symmetric pass over the node targets, the
// one-sided pass over the extra targets.  out: [M] (node targets first).
void launch_far_sym(const vp_ctx* ctx, const vp_nf* nf, const double* W, const double* f, double* out, void* ws,
                    cudaStream_t s, float2* f2out) {
    ensure_logtab();
    const SymPlan* p = nf->sym;
    const int64_t N = p->N, M = nf->M, m = M - N;
    const int sp = extra_splits(N, m, ctx->sm_count);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char* w = (char*)ws;
    double* rowbuf = (double*)w;
    w += al((size_t)p->max_band_units * SYM_TI * 8);
    double* colbuf = (double*)w;
    w += al((size_t)p->max_band_cols * 8);
    double* acc = (double*)w;
    w += al((size_t)N * 8);
    double* diag = (double*)w;
    w += al((size_t)N * 8);
    float* q = (float*)w;
    w += al((size_t)N * 2 * sizeof(float));
    double* xpart = (double*)w;
    const float* shi = nf->src_ff.hi;
    const float* slo = nf->src_ff.lo;
    k_prep_q_ff<1><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(W, f, N, 1, 0, q, f2out, nf->mesh->nq);
    for (size_t b = 0; b < p->bands.size(); b++) {
        const SymBand& bd = p->bands[b];
        if (bd.u1 > bd.u0)
            k_far_sym<<<(unsigned)(bd.u1 - bd.u0), SYM_THREADS, 0, s>>>(shi, slo, q, N, p->unit_I, p->unit_j0,
                                                                        p->unit_j1, p->coff, bd.u0, bd.c0, rowbuf,
                                                                        colbuf);
        const int64_t nodes = N - (int64_t)bd.tile0 * SYM_TI;
        k_far_sym_accum<<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(rowbuf, colbuf, p->ufirst, p->coff, N,
                                                                        bd.tile0, bd.tile1, bd.u0, bd.c0, b == 0,
                                                                        acc);
    }
    k_far_sym_diag<<<(unsigned)p->n_tiles, FF_THREADS, 0, s>>>(shi, slo, q, N, nf->d_tnode, diag);
    k_far_sym_combine<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(diag, acc, N, out);
    if (m > 0) {
        dim3 g((unsigned)((m + SYM_TI - 1) / SYM_TI), (unsigned)sp);
        k_far_extra<<<g, FF_THREADS, 0, s>>>(shi, slo, q, N, nf->tgt_ff.hi, nf->tgt_ff.lo, nf->d_tnode, M, sp, xpart);
        k_far_extra_reduce<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(xpart, sp, m, out + N);
    }
}

// Loads this unit's log table on the current device (vp_create).
cudaError_t far_sym_module_prepare() { return ensure_logtab(); }
