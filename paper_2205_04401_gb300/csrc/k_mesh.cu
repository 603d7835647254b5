// Mesh upload: counter-clockwise normalisation, Jacobians and quadrature
// nodes of every triangle (Theorem 3.1 with the affine map of Section 3.1).
#include "vp_internal.h"

namespace {

// One thread per triangle.  Node j = t*nq + k sits at
//   y = A + (xi_k (B - A) + eta_k (C - A)),  W_j = w_k J_T,
// evaluated with round-to-nearest operations in this order.
__global__ void k_mesh_nodes(const double* __restrict__ vxy, int64_t nv, const int32_t* __restrict__ tri, int64_t nt,
                             FarRuleDev fr, double* __restrict__ tv, double* __restrict__ J,
                             double* __restrict__ y, double* __restrict__ W, int32_t* flag) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
        atomicOr(flag, VP_DEV_ERR_BADIDX);
        return;
    }
    double Ax = vxy[2 * a], Ay = vxy[2 * a + 1];
    double Bx = vxy[2 * b], By = vxy[2 * b + 1];
    double Cx = vxy[2 * c], Cy = vxy[2 * c + 1];
    if (!isfinite(Ax) || !isfinite(Ay) || !isfinite(Bx) || !isfinite(By) || !isfinite(Cx) || !isfinite(Cy)) {
        atomicOr(flag, VP_DEV_ERR_NONFINITE);
        return;
    }
    double o = orient_rn(Ax, Ay, Bx, By, Cx, Cy);
    if (o < 0.0) {
        double sx = Bx, sy = By;
        Bx = Cx; By = Cy; Cx = sx; Cy = sy;
        o = -o;
    }
    if (!(o > 0.0)) {
        atomicOr(flag, VP_DEV_ERR_DEGEN);
        return;
    }
    double* v = tv + 6 * t;
    v[0] = Ax; v[1] = Ay; v[2] = Bx; v[3] = By; v[4] = Cx; v[5] = Cy;
    J[t] = o;
    const int nq = fr.nq;
    const double ex = rn_sub(Bx, Ax), ey = rn_sub(By, Ay);
    const double fx = rn_sub(Cx, Ax), fy = rn_sub(Cy, Ay);
    for (int k = 0; k < nq; k++) {
        const double xi = fr.x[k], eta = fr.y[k];
        int64_t j = t * nq + k;
        y[2 * j] = rn_add(Ax, rn_add(rn_mul(xi, ex), rn_mul(eta, fx)));
        y[2 * j + 1] = rn_add(Ay, rn_add(rn_mul(xi, ey), rn_mul(eta, fy)));
        W[j] = rn_mul(fr.w[k], o);
    }
}

}  // namespace

void launch_mesh_nodes(const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, FarRuleDev fr, double* tv,
                       double* J, double* y, double* W, int32_t* flag, cudaStream_t s) {
    if (nt <= 0) return;
    k_mesh_nodes<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(vxy, nv, tri, nt, fr, tv, J, y, W, flag);
}
