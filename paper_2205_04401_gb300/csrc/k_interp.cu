// Interpolation of the volume potential over a mesh (Section 3.5): on every
// element Delta of an interpolation mesh (straight, or curved through the
// blending map of Eq. for:blend) the Koornwinder expansion of u o rho of
// degree N_s is obtained from u at dim P_{N_s} interpolation nodes by the
// inverse interpolation matrix, and u(x) = I(rho^{-1}(x)).
//
// Kernels: the nodes of every element (rho of the reference nodes), the
// coefficients (one block per element and density: a dense dim P x dim P
// matrix-vector product with the inverse interpolation matrix), and the
// evaluation at arbitrary points (point location in a grid of element boxes
// with the exact predicates of App. A.5, rho^{-1} by the affine inverse or
// Newton's method, and the Koornwinder recurrences of Section 2.1).  All
// FP64: a staggered-mesh evaluation needs the potential to full accuracy.
#include "vp_internal.h"
#include "vp_curved.cuh"

namespace {

// sum_a coef[a] K_a(x, y) over the Koornwinder polynomials of degree <= N
// (Section 2.1), index a = n (n + 1)/2 + m:
//   K_mn = c_mn (1 - x)^m P_{n-m}^{(2m+1,0)}(2x - 1) P_m(2y/(1 - x) - 1),
// with (1 - x)^m P_m(...) from Legendre's recurrence in homogeneous form,
//   H_{m+1} = hA_m s H_m - hB_m (1 - x)^2 H_{m-1},   s = 2y + x - 1,
// and the Jacobi polynomials from their three-term recurrence,
//   P_{k+1} = (jA z + jB) P_k - jC P_{k-1},   z = 2x - 1,
// whose coefficients (and c_mn) come precomputed in `rec` (layout in
// interp_recurrences), so the loop has no division or square root.
__device__ double koornwinder_dot(int N, int nn, double x, double y, const double* __restrict__ rec,
                                  const double* __restrict__ coef) {
    const double* cn = rec;
    const double* jA = rec + nn;
    const double* jB = rec + 2 * nn;
    const double* jC = rec + 3 * nn;
    const double* hA = rec + 4 * nn;
    const double* hB = hA + (N + 1);
    const double w = 1.0 - x, s = 2.0 * y - w, w2 = w * w, z = 2.0 * x - 1.0;
    double Hm1 = 0.0, Hm = 1.0;   // H_{m-1}, H_m
    double acc = 0.0;
    for (int m = 0; m <= N; m++) {
        double pkm1 = 0.0, pk = Hm;   // H_m P_k, advanced by the Jacobi recurrence
        int a = m * (m + 1) / 2 + m;  // index of (n = m, m)
        for (int n = m; n <= N; n++) {
            acc = fma(coef[a] * cn[a], pk, acc);
            const double pn = fma(fma(jA[a], z, jB[a]), pk, -jC[a] * pkm1);
            pkm1 = pk;
            pk = pn;
            a += n + 1;               // (n + 1, m)
        }
        const double Hp = fma(hA[m] * s, Hm, -hB[m] * w2 * Hm1);
        Hm1 = Hm;
        Hm = Hp;
    }
    return acc;
}

// Nodes of every element: rho_T of the reference nodes (exact-rounding map,
// so straight elements reproduce A + xi (B - A) + eta (C - A)).
__global__ void k_interp_nodes(const double* __restrict__ tv, CurveDev cv, int64_t nt, const double* __restrict__ zx,
                               const double* __restrict__ zy, int nn, double* __restrict__ xy) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt * nn) return;
    const int64_t T = i / nn;
    const int k = (int)(i - T * nn);
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; q++) v[q] = tv[6 * T + q];
    geom_map_rn(v, curve_coef(cv, T), cv.K, zx[k], zy[k], xy + 2 * i, nullptr, nullptr);
}

// coef[d][T][a] = sum_b Vinv[a][b] u[d][T nn + b]; one block per (T, d).
__global__ void k_interp_coeffs(const double* __restrict__ Vinv, int nn, int64_t nt, const double* __restrict__ u,
                                double* __restrict__ coef) {
    extern __shared__ double su[];
    const int64_t T = blockIdx.x;
    const int64_t dd = blockIdx.y;
    const double* uT = u + (dd * nt + T) * nn;
    for (int b = threadIdx.x; b < nn; b += blockDim.x) su[b] = uT[b];
    __syncthreads();
    for (int a = threadIdx.x; a < nn; a += blockDim.x) {
        const double* row = Vinv + (int64_t)a * nn;
        double s0 = 0.0, s1 = 0.0;
        int b = 0;
        for (; b + 1 < nn; b += 2) {
            s0 = fma(row[b], su[b], s0);
            s1 = fma(row[b + 1], su[b + 1], s1);
        }
        if (b < nn) s0 = fma(row[b], su[b], s0);
        coef[(dd * nt + T) * nn + a] = s0 + s1;
    }
}

// Element boxes for point location (grown for curved elements by
// launch_curved_bbox).
__global__ void k_tri_bbox(const double* __restrict__ tv, int64_t nt, double* __restrict__ bbox) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* v = tv + 6 * t;
    bbox[4 * t] = fmin(v[0], fmin(v[2], v[4]));
    bbox[4 * t + 1] = fmin(v[1], fmin(v[3], v[5]));
    bbox[4 * t + 2] = fmax(v[0], fmax(v[2], v[4]));
    bbox[4 * t + 3] = fmax(v[1], fmax(v[3], v[5]));
}

__device__ __forceinline__ int32_t grid_cell(double v, double o, double h, int32_t n) {
    const double c = floor((v - o) / h);
    if (!(c >= 0.0)) return 0;                 // also NaN
    if (c >= (double)(n - 1)) return n - 1;
    return (int32_t)c;
}

// u at points: locate (lowest-index element of the point's cell that holds
// it), map back to the reference simplex, sum the expansion.  Points in no
// element get NaN and element -1.
__global__ void k_interp_eval(const double* __restrict__ tv, CurveDev cv, GridDev g, const double* __restrict__ pts,
                              int64_t m, int N, int nn, int64_t nt, const double* __restrict__ rec,
                              const double* __restrict__ coef, int d, double* __restrict__ out,
                              int32_t* __restrict__ elem) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double xx = pts[2 * i], xy = pts[2 * i + 1];
    int32_t T = -1;
    double v[6];
    if (xx >= g.ox && xy >= g.oy && xx <= g.ox + g.h * g.nx && xy <= g.oy + g.h * g.ny) {
        const int32_t c = grid_cell(xy, g.oy, g.h, g.ny) * g.nx + grid_cell(xx, g.ox, g.h, g.nx);
        for (int64_t k = g.cell_start[c]; k < g.cell_start[c + 1]; k++) {
            const int32_t Tk = g.cell_tri[k];
#pragma unroll
            for (int q = 0; q < 6; q++) v[q] = tv[6 * (int64_t)Tk + q];
            if (elem_contains_rn(v, curve_coef(cv, Tk), cv.K, xx, xy)) {
                T = Tk;
                break;
            }
        }
    }
    if (elem) elem[i] = T;
    if (T < 0) {
        for (int dd = 0; dd < d; dd++) out[(int64_t)dd * m + i] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double xi, eta;
    const double* ax = curve_coef(cv, T);
    if (ax) {
        geom_inverse_rn(v, ax, cv.K, xx, xy, &xi, &eta);
    } else {
        const double ex = v[2] - v[0], ey = v[3] - v[1], fx = v[4] - v[0], fy = v[5] - v[1];
        const double qx = xx - v[0], qy = xy - v[1];
        const double J = ex * fy - ey * fx;
        xi = (qx * fy - qy * fx) / J;
        eta = (ex * qy - ey * qx) / J;
    }
    for (int dd = 0; dd < d; dd++)
        out[(int64_t)dd * m + i] = koornwinder_dot(N, nn, xi, eta, rec, coef + ((int64_t)dd * nt + T) * nn);
}

}  // namespace

void launch_interp_nodes(const double* tv, CurveDev cv, int64_t nt, const double* zx, const double* zy, int nn,
                         double* xy, cudaStream_t s) {
    const int64_t n = nt * nn;
    if (n > 0) k_interp_nodes<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tv, cv, nt, zx, zy, nn, xy);
}

void launch_interp_coeffs(const double* Vinv, int nn, int64_t nt, int d, const double* u, double* coef,
                          cudaStream_t s) {
    if (nt <= 0 || d <= 0) return;
    const int threads = nn > 128 ? 256 : 128;
    k_interp_coeffs<<<dim3((unsigned)nt, (unsigned)d), threads, nn * sizeof(double), s>>>(Vinv, nn, nt, u, coef);
}

void launch_tri_bbox(const double* tv, int64_t nt, double* bbox, cudaStream_t s) {
    if (nt > 0) k_tri_bbox<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(tv, nt, bbox);
}

void launch_interp_eval(const double* tv, CurveDev cv, GridDev g, const double* pts, int64_t m, int N, int nn,
                        int64_t nt, const double* rec, const double* coef, int d, double* out, int32_t* elem,
                        cudaStream_t s) {
    if (m > 0)
        k_interp_eval<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(tv, cv, g, pts, m, N, nn, nt, rec, coef, d, out,
                                                                   elem);
}
