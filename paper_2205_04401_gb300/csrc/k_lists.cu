// Near-field lists (Section 4.1) and point location (Appendix A.5) on a
// uniform grid.  Every triangle is binned into the grid cells covered by the
// bounding box of its three edge ellipses (the paper uses a quadtree over
// bounding-box corners; a uniform grid is the GPU-friendly equivalent).  Each
// target then scans the triangles of its own cell, in ascending index order,
// with the exact FP64 predicates, so the lists come out sorted and identical
// to a brute-force scan over all triangles.
#include "vp_internal.h"

namespace {

__device__ __forceinline__ int32_t cell_coord(double v, double o, double h, int32_t n) {
    double c = floor((v - o) / h);
    if (!(c >= 0.0)) return 0;          // also catches NaN
    if (c >= (double)(n - 1)) return n - 1;
    return (int32_t)c;
}

// R_T and a conservative bounding box of T united with its three ellipses.
__global__ void k_tri_geom(const double* __restrict__ tv, const double* __restrict__ J, int64_t nt, double what, int N,
                           double eps, double cn, double* __restrict__ R, double* __restrict__ bbox) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* v = tv + 6 * t;
    double r = ellipse_R_rn(what, J[t], eps, cn);
    R[t] = r;
    double rho0 = r > 1.0 ? pow(r, 1.0 / N) : 1.0;
    double x0 = fmin(v[0], fmin(v[2], v[4])), x1 = fmax(v[0], fmax(v[2], v[4]));
    double y0 = fmin(v[1], fmin(v[3], v[5])), y1 = fmax(v[1], fmax(v[3], v[5]));
    for (int e = 0; e < 3; e++) {
        double px = v[2 * e], py = v[2 * e + 1];
        double qx = v[(2 * e + 2) % 6], qy = v[(2 * e + 3) % 6];
        double L = sqrt((qx - px) * (qx - px) + (qy - py) * (qy - py));
        double a = 0.25 * L * (rho0 + 1.0 / rho0);
        double mx = 0.5 * (px + qx), my = 0.5 * (py + qy);
        a = a * (1.0 + 1e-9) + 1e-15 * (fabs(mx) + fabs(my) + L);
        x0 = fmin(x0, mx - a); x1 = fmax(x1, mx + a);
        y0 = fmin(y0, my - a); y1 = fmax(y1, my + a);
    }
    bbox[4 * t] = x0; bbox[4 * t + 1] = y0; bbox[4 * t + 2] = x1; bbox[4 * t + 3] = y1;
}

// Single-block min/max over n boxes (stride 4: x0 y0 x1 y1) or points
// (stride 2: x y, used as both corners).
__global__ void k_bbox_reduce(const double* __restrict__ b, int64_t n, int stride, double* out4) {
    double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double* p = b + stride * i;
        x0 = fmin(x0, p[0]); y0 = fmin(y0, p[1]);
        x1 = fmax(x1, p[stride == 4 ? 2 : 0]); y1 = fmax(y1, p[stride == 4 ? 3 : 1]);
    }
    __shared__ double s[4][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = x0; s[1][w] = y0; s[2][w] = x1; s[3][w] = y1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            x0 = fmin(x0, s[0][i]); y0 = fmin(y0, s[1][i]); x1 = fmax(x1, s[2][i]); y1 = fmax(y1, s[3][i]);
        }
        out4[0] = x0; out4[1] = y0; out4[2] = x1; out4[3] = y1;
    }
}

__global__ void k_tri_cell_count(const double* __restrict__ bbox, int64_t nt, GridDev g, int32_t* cnt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* b = bbox + 4 * t;
    int32_t ix0 = cell_coord(b[0], g.ox, g.h, g.nx), ix1 = cell_coord(b[2], g.ox, g.h, g.nx);
    int32_t iy0 = cell_coord(b[1], g.oy, g.h, g.ny), iy1 = cell_coord(b[3], g.oy, g.h, g.ny);
    for (int32_t iy = iy0; iy <= iy1; iy++)
        for (int32_t ix = ix0; ix <= ix1; ix++) atomicAdd(&cnt[(int64_t)iy * g.nx + ix], 1);
}

__global__ void k_tri_cell_fill(const double* __restrict__ bbox, int64_t nt, GridDev g, int64_t* cursor,
                                int32_t* __restrict__ cell_tri) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* b = bbox + 4 * t;
    int32_t ix0 = cell_coord(b[0], g.ox, g.h, g.nx), ix1 = cell_coord(b[2], g.ox, g.h, g.nx);
    int32_t iy0 = cell_coord(b[1], g.oy, g.h, g.ny), iy1 = cell_coord(b[3], g.oy, g.h, g.ny);
    for (int32_t iy = iy0; iy <= iy1; iy++)
        for (int32_t ix = ix0; ix <= ix1; ix++) {
            unsigned long long p = atomicAdd((unsigned long long*)&cursor[(int64_t)iy * g.nx + ix], 1ull);
            cell_tri[p] = (int32_t)t;
        }
}

// Block per cell: bitonic sort of the cell's triangle indices in shared
// memory (size = next power of two >= the largest cell, given by the host).
__global__ void k_cell_sort(GridDev g, int64_t ncell, int32_t cap, int32_t* __restrict__ cell_tri, int32_t* flag) {
    extern __shared__ int32_t sm[];
    int64_t c = blockIdx.x;
    if (c >= ncell) return;
    int64_t s0 = g.cell_start[c], s1 = g.cell_start[c + 1];
    int32_t n = (int32_t)(s1 - s0);
    if (n <= 1) return;
    if (n > cap) {
        if (threadIdx.x == 0) atomicOr(flag, VP_DEV_ERR_CELL);
        return;
    }
    int32_t S = 1;
    while (S < n) S <<= 1;
    for (int32_t i = threadIdx.x; i < S; i += blockDim.x) sm[i] = i < n ? cell_tri[s0 + i] : INT32_MAX;
    __syncthreads();
    for (int32_t k = 2; k <= S; k <<= 1) {
        for (int32_t j = k >> 1; j > 0; j >>= 1) {
            for (int32_t i = threadIdx.x; i < S; i += blockDim.x) {
                int32_t p = i ^ j;
                if (p > i) {
                    int32_t a = sm[i], b = sm[p];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { sm[i] = b; sm[p] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) cell_tri[s0 + i] = sm[i];
}

// Targets: the N nodes (if requested) then the m extra points.
__global__ void k_targets_init(const double* __restrict__ ynode, int64_t N, int nq, int node_targets,
                               const double* __restrict__ extra, int64_t m, double* __restrict__ txy,
                               int32_t* __restrict__ tnode, int32_t* __restrict__ tself) {
    int64_t nn = node_targets ? N : 0;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn + m) return;
    if (i < nn) {
        txy[2 * i] = ynode[2 * i];
        txy[2 * i + 1] = ynode[2 * i + 1];
        tnode[i] = (int32_t)i;
        tself[i] = (int32_t)(i / nq);
    } else {
        int64_t e = i - nn;
        txy[2 * i] = extra[2 * e];
        txy[2 * i + 1] = extra[2 * e + 1];
        tnode[i] = -1;
        tself[i] = -1;
    }
}

__global__ void k_target_cells(const double* __restrict__ txy, int64_t M, GridDev g, int32_t* __restrict__ tcell,
                               int32_t* __restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int32_t ix = cell_coord(txy[2 * i], g.ox, g.h, g.nx), iy = cell_coord(txy[2 * i + 1], g.oy, g.h, g.ny);
    int32_t c = iy * g.nx + ix;
    tcell[i] = c;
    atomicAdd(&cnt[c], 1);
}

__global__ void k_target_order(const int32_t* __restrict__ tcell, int64_t M, int64_t* cursor, int32_t* __restrict__ order) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    unsigned long long p = atomicAdd((unsigned long long*)&cursor[tcell[i]], 1ull);
    order[p] = (int32_t)i;
}

// S(x) for targets that are not nodes: the first (lowest-index) triangle of
// the cell list whose three orientation tests are >= 0.
__global__ void k_locate(const double* __restrict__ tv, const double* __restrict__ txy, const int32_t* __restrict__ order,
                         const int32_t* __restrict__ tcell, int64_t M, GridDev g, int32_t* __restrict__ tself) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int32_t t = order[i];
    if (tself[t] >= 0) return;
    double xx = txy[2 * t], xy = txy[2 * t + 1];
    int32_t c = tcell[t];
    int64_t s0 = g.cell_start[c], s1 = g.cell_start[c + 1];
    for (int64_t k = s0; k < s1; k++) {
        int32_t T = g.cell_tri[k];
        double v[6];
#pragma unroll
        for (int q = 0; q < 6; q++) v[q] = tv[6 * (int64_t)T + q];
        if (tri_contains_rn(v, xx, xy)) {
            tself[t] = T;
            return;
        }
    }
}

// Count (row == nullptr) or fill the target-major list of each target:
// kind 1 for S(x), kind 0 for T != S(x) whose ellipses hold x.  With a
// cache, the counting pass also keeps up to `cap` entries per target (T, and
// the kind in the top bit) and the filling pass copies them instead of
// testing again; targets with more entries are tested again.
__global__ void k_list_pass(const double* __restrict__ tv, const double* __restrict__ R, int N,
                            const double* __restrict__ txy, const int32_t* __restrict__ tself,
                            const int32_t* __restrict__ order, const int32_t* __restrict__ tcell, int64_t M, GridDev g,
                            int32_t* __restrict__ count, const int64_t* __restrict__ row, int32_t* __restrict__ ptri,
                            int32_t* __restrict__ ptgt, uint8_t* __restrict__ pkind, uint32_t* __restrict__ cache,
                            int cap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int32_t t = order[i];
    if (row && cache) {
        const int64_t o0 = row[t];
        const int32_t cnt = (int32_t)(row[t + 1] - o0);
        if (cnt <= cap) {
            const uint32_t* ce = cache + (int64_t)t * cap;
            for (int32_t k = 0; k < cnt; k++) {
                const uint32_t e = ce[k];
                ptri[o0 + k] = (int32_t)(e & 0x7fffffffu);
                ptgt[o0 + k] = t;
                pkind[o0 + k] = (uint8_t)(e >> 31);
            }
            return;
        }
    }
    double xx = txy[2 * t], xy = txy[2 * t + 1];
    int32_t S = tself[t];
    int32_t c = tcell[t];
    int64_t s0 = g.cell_start[c], s1 = g.cell_start[c + 1];
    int64_t out = row ? row[t] : 0;
    int32_t n = 0;
    for (int64_t k = s0; k < s1; k++) {
        int32_t T = g.cell_tri[k];
        int kind;
        if (T == S) kind = 1;
        else {
            double v[6];
#pragma unroll
            for (int q = 0; q < 6; q++) v[q] = tv[6 * (int64_t)T + q];
            kind = tri_near_fast(v, xx, xy, N, R[T]) ? 0 : -1;
        }
        if (kind >= 0) {
            if (row) {
                ptri[out + n] = T;
                ptgt[out + n] = t;
                pkind[out + n] = (uint8_t)kind;
            } else if (cache && n < cap) {
                cache[(int64_t)t * cap + n] = (uint32_t)T | ((uint32_t)kind << 31);
            }
            n++;
        }
    }
    if (!row) count[t] = n;
}

}  // namespace

void launch_tri_geom(const double* tv, const double* J, int64_t nt, double what, int N, double eps, double cn,
                     double* R, double* bbox, cudaStream_t s) {
    if (nt > 0) k_tri_geom<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(tv, J, nt, what, N, eps, cn, R, bbox);
}

void launch_bbox_reduce(const double* bbox, int64_t n, int stride, double* out4, cudaStream_t s) {
    k_bbox_reduce<<<1, 1024, 0, s>>>(bbox, n, stride, out4);
}

void launch_tri_cell_count(const double* bbox, int64_t nt, GridDev g, int32_t* cnt, cudaStream_t s) {
    if (nt > 0) k_tri_cell_count<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(bbox, nt, g, cnt);
}

void launch_tri_cell_fill(const double* bbox, int64_t nt, GridDev g, int64_t* cursor, int32_t* cell_tri,
                          cudaStream_t s) {
    if (nt > 0) k_tri_cell_fill<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(bbox, nt, g, cursor, cell_tri);
}

void launch_cell_sort(GridDev g, int64_t ncell, int32_t max_count, int32_t* cell_tri, int32_t* flag, cudaStream_t s) {
    int32_t S = 1;
    while (S < max_count) S <<= 1;
    size_t smem = (size_t)S * sizeof(int32_t);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_cell_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ncell > 0) k_cell_sort<<<(unsigned)ncell, 256, smem, s>>>(g, ncell, S, cell_tri, flag);
}

void launch_targets_init(const double* ynode, int64_t N, int nq, int node_targets, const double* extra, int64_t m,
                         double* txy, int32_t* tnode, int32_t* tself, cudaStream_t s) {
    int64_t M = (node_targets ? N : 0) + m;
    if (M > 0)
        k_targets_init<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(ynode, N, nq, node_targets, extra, m, txy, tnode, tself);
}

void launch_target_cells(const double* txy, int64_t M, GridDev g, int32_t* tcell, int32_t* cnt, cudaStream_t s) {
    if (M > 0) k_target_cells<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(txy, M, g, tcell, cnt);
}

void launch_target_order(const int32_t* tcell, int64_t M, int64_t* cursor, int32_t* order, cudaStream_t s) {
    if (M > 0) k_target_order<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(tcell, M, cursor, order);
}

void launch_locate(const double* tv, const double* txy, const int32_t* order, const int32_t* tcell, int64_t M,
                   GridDev g, int32_t* tself, cudaStream_t s) {
    if (M > 0) k_locate<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(tv, txy, order, tcell, M, g, tself);
}

void launch_list_pass(const double* tv, const double* R, int N, const double* txy, const int32_t* tself,
                      const int32_t* order, const int32_t* tcell, int64_t M, GridDev g, int32_t* count,
                      const int64_t* row, int32_t* ptri, int32_t* ptgt, uint8_t* pkind, uint32_t* cache, int cap,
                      cudaStream_t s) {
    if (M > 0)
        k_list_pass<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(tv, R, N, txy, tself, order, tcell, M, g, count, row,
                                                                ptri, ptgt, pkind, cache, cap);
}
