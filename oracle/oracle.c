/*
 * CPU oracle for the 2-D volume potential  u(x) = int_Omega (1/2pi) log|x-y| f(y) dA
 * evaluated by the subtract-and-add scheme of Shen & Serkh (arXiv 2205.04401).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain FP64 C, one loop per step of the paper,
 * no blocking or reordering beyond what the paper states.  Compiled with
 * -O2 -ffp-contract=off so that no multiply-add is fused.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark call it; the
 * library never does.
 *
 * Conventions (shared with the library only through the paper's definitions):
 *   reference simplex  {(x,y): x>=0, y>=0, x+y<=1};  map of triangle (A,B,C):
 *   rho_T(xi,eta) = A + xi (B-A) + eta (C-A);  J_T = (B-A) x (C-A) > 0 (CCW).
 *   G(x,y) = log|x-y| / (2 pi).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NB 15 /* dim P_4 */
#define TWO_PI 6.283185307179586476925286766559
#define MAXQ 1024

typedef struct {
    /* far rule (Section 3.2): nq nodes on the reference simplex */
    int nq, far_degree;
    double fx[MAXQ], fy[MAXQ], fw[MAXQ];
    double far_what, far_cn;
    /* near rule (Section 3.3), applied on every leaf of the subdivision */
    int nn, near_degree;
    double nx[MAXQ], ny[MAXQ], nw[MAXQ];
    double near_what, near_cn;
    /* generalized Gaussian rule in the radial variable (Section 3.4) */
    int ng;
    double gr[16], gw[16];
    /* Gauss-Legendre panel rule in the arc-length variable (Section 3.4) */
    int nl;
    double lx[32], lw[32];
    /* orthonormal P_4 basis on the reference simplex: K = Linv * [P_a(2x-1) P_b(2y-1)] */
    int bidx_a[NB], bidx_b[NB];
    double Linv[NB][NB];
    double eps;
    int depth_cap;
} or_params;

/* ------------------------------------------------------------ basics ---- */
static double kernelG(double x0, double x1, double y0, double y1) {
    double dx = x0 - y0, dy = x1 - y1;
    return 0.5 * log(dx * dx + dy * dy) / TWO_PI;
}

/* orientation o_PQ(X) = (Q-P) x (X-P), evaluated in this order, no FMA */
static double orient(double px, double py, double qx, double qy, double xx, double xy) {
    double a = (qx - px) * (xy - py);
    double b = (qy - py) * (xx - px);
    return a - b;
}

/* orthonormal basis values K_alpha(xi, eta), alpha = 0..14 */
static void basis(const or_params* P, double xi, double eta, double* K) {
    double la[5], lb[5];
    double u = 2.0 * xi - 1.0, v = 2.0 * eta - 1.0;
    la[0] = 1.0; la[1] = u;
    lb[0] = 1.0; lb[1] = v;
    for (int n = 1; n < 4; n++) {
        la[n + 1] = ((2.0 * n + 1.0) * u * la[n] - n * la[n - 1]) / (n + 1.0);
        lb[n + 1] = ((2.0 * n + 1.0) * v * lb[n] - n * lb[n - 1]) / (n + 1.0);
    }
    double raw[NB];
    for (int i = 0; i < NB; i++) raw[i] = la[P->bidx_a[i]] * lb[P->bidx_b[i]];
    for (int i = 0; i < NB; i++) {
        double s = 0.0;
        for (int j = 0; j <= i; j++) s += P->Linv[i][j] * raw[j];
        K[i] = s;
    }
}

/* --------------------------------------------------- nodes (Thm 3.1) ---- */
/* Triangles are made counter-clockwise by swapping B and C when (B-A)x(C-A) < 0.
 * Node j = T*nq + k sits at rho_T(xi_k, eta_k) with weight w_k * J_T. */
int or_nodes(const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, const or_params* P,
             int32_t* tri_ccw, double* yxy, double* W, double* J) {
    for (int64_t t = 0; t < nt; t++) {
        int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) return -1;
        double o = orient(vxy[2 * a], vxy[2 * a + 1], vxy[2 * b], vxy[2 * b + 1], vxy[2 * c], vxy[2 * c + 1]);
        if (o < 0) { int32_t s = b; b = c; c = s; o = -o; }
        if (!(o > 0)) return -2;
        tri_ccw[3 * t] = a; tri_ccw[3 * t + 1] = b; tri_ccw[3 * t + 2] = c;
        J[t] = o;
        double Ax = vxy[2 * a], Ay = vxy[2 * a + 1];
        double ex = vxy[2 * b] - Ax, ey = vxy[2 * b + 1] - Ay;
        double fx = vxy[2 * c] - Ax, fy = vxy[2 * c + 1] - Ay;
        for (int k = 0; k < P->nq; k++) {
            int64_t j = t * P->nq + k;
            yxy[2 * j] = Ax + (P->fx[k] * ex + P->fy[k] * fx);
            yxy[2 * j + 1] = Ay + (P->fx[k] * ey + P->fy[k] * fy);
            W[j] = P->fw[k] * o;
        }
    }
    return 0;
}

/* ------------------------------------------- point location (App. A.5) -- */
/* S(x): the lowest-index triangle whose three orientation tests are >= 0. */
int64_t or_locate_one(const double* vxy, const int32_t* tri, int64_t nt, double x, double y) {
    for (int64_t t = 0; t < nt; t++) {
        const int32_t* v = tri + 3 * t;
        double Ax = vxy[2 * v[0]], Ay = vxy[2 * v[0] + 1];
        double Bx = vxy[2 * v[1]], By = vxy[2 * v[1] + 1];
        double Cx = vxy[2 * v[2]], Cy = vxy[2 * v[2] + 1];
        if (orient(Ax, Ay, Bx, By, x, y) >= 0 && orient(Bx, By, Cx, Cy, x, y) >= 0 &&
            orient(Cx, Cy, Ax, Ay, x, y) >= 0)
            return t;
    }
    return -1;
}

void or_locate(const double* vxy, const int32_t* tri, int64_t nt, const double* pts, int64_t m, int32_t* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; i++) out[i] = (int32_t)or_locate_one(vxy, tri, nt, pts[2 * i], pts[2 * i + 1]);
}

/* ------------------------------------- far sum (Section 3.6, all nodes) -- */
/* u_far(x_t) = sum_j W_j f_j G(x_t, y_j), skipping the target's own node.
 * Neumaier-compensated FP64 sum.  f is [d][N], out is [d][M]. */
void or_far(const double* yxy, const double* W, int64_t N, const double* f, int d,
            const double* txy, const int64_t* tnode, int64_t M, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < M; t++) {
        for (int k = 0; k < d; k++) {
            double s = 0.0, c = 0.0;
            for (int64_t j = 0; j < N; j++) {
                if (j == tnode[t]) continue;
                double term = W[j] * f[(int64_t)k * N + j] * kernelG(txy[2 * t], txy[2 * t + 1], yxy[2 * j], yxy[2 * j + 1]);
                double u = s + term;
                if (fabs(s) >= fabs(term)) c += (s - u) + term; else c += (term - u) + s;
                s = u;
            }
            out[(int64_t)k * M + t] = s + c;
        }
    }
}

/* --------------------------------- near-field predicate (Section 4.1) ---- */
/* Edge (P,Q), target X: the open Bernstein ellipse with foci P, Q and
 * parameter rho0 = R^(1/N) (Eq. rho0 with R = w J / (eps C_N)) contains X iff
 * rho_X^N < R, where rho_X = s + sqrt(s^2 - 1) and s = (|X-P| + |X-Q|)/|Q-P|.
 * rho_X^N is a left-to-right product (no pow). */
static int edge_near(double px, double py, double qx, double qy, double xx, double xy, int N, double R) {
    double ex = qx - px, ey = qy - py;
    double L = sqrt(ex * ex + ey * ey);
    double ax = xx - px, ay = xy - py, bx = xx - qx, by = xy - qy;
    double s = (sqrt(ax * ax + ay * ay) + sqrt(bx * bx + by * by)) / L;
    double t = s * s - 1.0;
    if (t < 0.0) t = 0.0;
    double rho = s + sqrt(t);
    double p = rho;
    for (int i = 1; i < N; i++) p = p * rho;
    return p < R;
}

static int tri_near(double Ax, double Ay, double Bx, double By, double Cx, double Cy,
                    double xx, double xy, int N, double R) {
    return edge_near(Ax, Ay, Bx, By, xx, xy, N, R) || edge_near(Bx, By, Cx, Cy, xx, xy, N, R) ||
           edge_near(Cx, Cy, Ax, Ay, xx, xy, N, R);
}

/* R_T = (w * J_T) / (eps * C_N) */
static double ellipse_R(double what, double J, double eps, double cn) { return (what * J) / (eps * cn); }

/* Per-target lists (Definition 3.3): S(x) and N(x) = {T != S(x): x in E_T}.
 * Output row of target i: triangles ascending, kind 1 = self, 0 = near.
 * Pass out_tri == NULL to count only. */
void or_lists(const double* vxy, const int32_t* tri, const double* J, int64_t nt, const or_params* P,
              const double* txy, const int32_t* tself, int64_t m, int64_t* count,
              const int64_t* row_ptr, int32_t* out_tri, uint8_t* out_kind) {
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < m; i++) {
        double xx = txy[2 * i], xy = txy[2 * i + 1];
        int64_t c = 0;
        for (int64_t t = 0; t < nt; t++) {
            const int32_t* v = tri + 3 * t;
            int kind = -1;
            if (t == tself[i]) kind = 1;
            else if (tri_near(vxy[2 * v[0]], vxy[2 * v[0] + 1], vxy[2 * v[1]], vxy[2 * v[1] + 1],
                              vxy[2 * v[2]], vxy[2 * v[2] + 1], xx, xy, P->far_degree,
                              ellipse_R(P->far_what, J[t], P->eps, P->far_cn)))
                kind = 0;
            if (kind >= 0) {
                if (out_tri) { out_tri[row_ptr[i] + c] = (int32_t)t; out_kind[row_ptr[i] + c] = (uint8_t)kind; }
                c++;
            }
        }
        count[i] = c;
    }
}

/* Test hook: the near predicate alone for (point, triangle) pairs. */
void or_near_pred(const double* vxy, const int32_t* tri, const double* J, const or_params* P,
                  const double* pts, const int64_t* tids, int64_t n, uint8_t* out) {
    for (int64_t i = 0; i < n; i++) {
        const int32_t* v = tri + 3 * tids[i];
        out[i] = (uint8_t)tri_near(vxy[2 * v[0]], vxy[2 * v[0] + 1], vxy[2 * v[1]], vxy[2 * v[1] + 1],
                                   vxy[2 * v[2]], vxy[2 * v[2] + 1], pts[2 * i], pts[2 * i + 1],
                                   P->far_degree, ellipse_R(P->far_what, J[tids[i]], P->eps, P->far_cn));
    }
}

/* ---------------------- correction weights: moments -> nodal weights ---- */
/* The density on T is its discrete L2 projection onto P_4 with the far rule
 * (exact Gram matrix because the rule has degree >= 8):
 *   Pi f (xi) = sum_k f_k w_k sum_a K_a(xi_k) K_a(xi).
 * With moments m_a = int_T G(x, y) K_a(rho_T^{-1} y) dA, the correction for
 * node k of T is  C_k = w_k sum_a K_a(xi_k) m_a - [k != own] W_k G(x, y_k). */
static void moments_to_weights(const or_params* P, const double* m, double J, double xx, double xy,
                               const double* A, const double* B, const double* C, int own, double* out) {
    for (int k = 0; k < P->nq; k++) {
        double K[NB];
        basis(P, P->fx[k], P->fy[k], K);
        double s = 0.0;
        for (int a = 0; a < NB; a++) s += K[a] * m[a];
        double val = P->fw[k] * s;
        if (k != own) {
            double yx = A[0] + (P->fx[k] * (B[0] - A[0]) + P->fy[k] * (C[0] - A[0]));
            double yy = A[1] + (P->fx[k] * (B[1] - A[1]) + P->fy[k] * (C[1] - A[1]));
            val -= P->fw[k] * J * kernelG(xx, xy, yx, yy);
        }
        out[k] = val;
    }
}

/* ------------------------ near interaction: adaptive subdivision (3.3) -- */
/* Subdivide the reference simplex by 4-way midpoint splits until each leaf S
 * has the target outside S and outside every edge ellipse of S (stop test of
 * Section 4.1 with the near rule's order N_n and R_S = w_n J_S / (eps C_Nn));
 * on each leaf apply the near rule (Eq. sum_near).  J_S = J_T 4^-depth. */
typedef struct { double v[6]; int depth; } subtri;

static void near_moments(const or_params* P, const double* A, const double* B, const double* C, double J,
                         double xx, double xy, double* m, int64_t* leaves, int64_t* capped) {
    subtri stack[4 * 64 + 8];
    int sp = 0;
    stack[sp].v[0] = 0; stack[sp].v[1] = 0; stack[sp].v[2] = 1; stack[sp].v[3] = 0;
    stack[sp].v[4] = 0; stack[sp].v[5] = 1; stack[sp].depth = 0; sp++;
    double ex = B[0] - A[0], ey = B[1] - A[1], fx = C[0] - A[0], fy = C[1] - A[1];
    for (int a = 0; a < NB; a++) m[a] = 0.0;
    while (sp > 0) {
        subtri S = stack[--sp];
        double ph[6];
        for (int i = 0; i < 3; i++) {
            ph[2 * i] = A[0] + (S.v[2 * i] * ex + S.v[2 * i + 1] * fx);
            ph[2 * i + 1] = A[1] + (S.v[2 * i] * ey + S.v[2 * i + 1] * fy);
        }
        double JS = ldexp(J, -2 * S.depth);
        int inside = orient(ph[0], ph[1], ph[2], ph[3], xx, xy) >= 0 && orient(ph[2], ph[3], ph[4], ph[5], xx, xy) >= 0 &&
                     orient(ph[4], ph[5], ph[0], ph[1], xx, xy) >= 0;
        int stop = !inside && !tri_near(ph[0], ph[1], ph[2], ph[3], ph[4], ph[5], xx, xy, P->near_degree,
                                        ellipse_R(P->near_what, JS, P->eps, P->near_cn));
        if (!stop && S.depth >= P->depth_cap) { stop = 1; (*capped)++; }
        if (stop) {
            (*leaves)++;
            for (int j = 0; j < P->nn; j++) {
                double xi = S.v[0] + (P->nx[j] * (S.v[2] - S.v[0]) + P->ny[j] * (S.v[4] - S.v[0]));
                double eta = S.v[1] + (P->nx[j] * (S.v[3] - S.v[1]) + P->ny[j] * (S.v[5] - S.v[1]));
                double yx = A[0] + (xi * ex + eta * fx);
                double yy = A[1] + (xi * ey + eta * fy);
                double g = kernelG(xx, xy, yx, yy) * P->nw[j] * JS;
                double K[NB];
                basis(P, xi, eta, K);
                for (int a = 0; a < NB; a++) m[a] += g * K[a];
            }
        } else {
            double m01x = 0.5 * (S.v[0] + S.v[2]), m01y = 0.5 * (S.v[1] + S.v[3]);
            double m12x = 0.5 * (S.v[2] + S.v[4]), m12y = 0.5 * (S.v[3] + S.v[5]);
            double m20x = 0.5 * (S.v[4] + S.v[0]), m20y = 0.5 * (S.v[5] + S.v[1]);
            double ch[4][6] = {{S.v[0], S.v[1], m01x, m01y, m20x, m20y},
                               {m01x, m01y, S.v[2], S.v[3], m12x, m12y},
                               {m20x, m20y, m12x, m12y, S.v[4], S.v[5]},
                               {m12x, m12y, m20x, m20y, m01x, m01y}};
            for (int c = 0; c < 4; c++) {
                memcpy(stack[sp].v, ch[c], sizeof(ch[c]));
                stack[sp].depth = S.depth + 1;
                sp++;
            }
        }
    }
}

/* ------------------ self interaction: radius-arclength coordinates (3.4) */
/* Split T into the three triangles (x, P, Q) over its edges (Section 3.4).
 * On each: int_0^L int_0^1 log(r0(s) r) F(y(r,s)) r h dr ds, with h the
 * distance from x to the line PQ (Observation: constant for a straight side),
 * the generalized Gaussian rule in r and Gauss-Legendre panels in s graded
 * toward s~ = argmin |x - gamma(s)| (clamped to [0, L]):
 *   N = min{n >= 0 : 2^-n s~ < |x - gamma(s~)|} panels + 1 on [0, s~],
 *   M = min{n >= 0 : 2^-n (L - s~) < |x - gamma(s~)|} panels + 1 on [s~, L]. */
static int dyadic_count(double len, double dist) {
    int n = 0;
    while (ldexp(len, -n) >= dist) n++;
    return n;
}

static void self_moments(const or_params* P, const double* A, const double* B, const double* C, double J,
                         double xx, double xy, double* m, int64_t* panels) {
    const double* V[3] = {A, B, C};
    double ex = B[0] - A[0], ey = B[1] - A[1], fx = C[0] - A[0], fy = C[1] - A[1];
    for (int a = 0; a < NB; a++) m[a] = 0.0;
    for (int e = 0; e < 3; e++) {
        const double* Pp = V[e];
        const double* Qp = V[(e + 1) % 3];
        double dx = Qp[0] - Pp[0], dy = Qp[1] - Pp[1];
        double L = sqrt(dx * dx + dy * dy);
        if (L == 0.0) continue;
        double h = fabs(dx * (xy - Pp[1]) - dy * (xx - Pp[0])) / L;
        if (h == 0.0) continue;
        double st = (dx * (xx - Pp[0]) + dy * (xy - Pp[1])) / L;
        if (st < 0.0) st = 0.0;
        if (st > L) st = L;
        double fxp = Pp[0] + (st / L) * dx, fyp = Pp[1] + (st / L) * dy;
        double delta = sqrt((xx - fxp) * (xx - fxp) + (xy - fyp) * (xy - fyp));
        /* panel endpoints */
        double bnd[2][130];
        int nb[2] = {0, 0};
        if (st > 0.0) {
            int N = dyadic_count(st, delta);
            bnd[0][nb[0]++] = 0.0;
            for (int i = 1; i <= N; i++) bnd[0][nb[0]++] = (1.0 - ldexp(1.0, -i)) * st;
            bnd[0][nb[0]++] = st;
        }
        if (st < L) {
            int Mm = dyadic_count(L - st, delta);
            bnd[1][nb[1]++] = L;
            for (int i = 1; i <= Mm; i++) bnd[1][nb[1]++] = L - (1.0 - ldexp(1.0, -i)) * (L - st);
            bnd[1][nb[1]++] = st;
        }
        for (int side = 0; side < 2; side++) {
            for (int p = 0; p + 1 < nb[side]; p++) {
                double s0 = bnd[side][p], s1 = bnd[side][p + 1];
                (*panels)++;
                for (int l = 0; l < P->nl; l++) {
                    double s = s0 + (s1 - s0) * P->lx[l];
                    double ws = (s1 - s0) * P->lw[l];
                    if (ws < 0) ws = -ws;
                    double gx = Pp[0] + (s / L) * dx, gy = Pp[1] + (s / L) * dy;
                    double r0 = sqrt((gx - xx) * (gx - xx) + (gy - xy) * (gy - xy));
                    for (int j = 0; j < P->ng; j++) {
                        double r = P->gr[j];
                        double yx = xx + r * (gx - xx), yy = xy + r * (gy - xy);
                        /* rho_T^{-1}(y) */
                        double qx = yx - A[0], qy = yy - A[1];
                        double xi = (qx * fy - qy * fx) / J;
                        double eta = (ex * qy - ey * qx) / J;
                        double K[NB];
                        basis(P, xi, eta, K);
                        double g = (log(r0) + log(r)) / TWO_PI * ws * h * P->gw[j];
                        for (int a = 0; a < NB; a++) m[a] += g * K[a];
                    }
                }
            }
        }
    }
}

/* Correction weights for (target, triangle, kind) pairs.
 * own[i] = node index k within T of the target (node targets on their own
 * triangle), else -1.  out is [npairs][nq]; stats[i] = leaves (near) or
 * s-panels (self); capped counts leaves stopped by the depth cap. */
void or_weights(const double* vxy, const int32_t* tri, const double* J, const or_params* P,
                const double* txy, const int64_t* pt, const int32_t* ptri, const uint8_t* pkind,
                const int32_t* pown, int64_t npairs, double* out, int64_t* stats, int64_t* capped_total) {
    int64_t capped_sum = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : capped_sum)
    for (int64_t i = 0; i < npairs; i++) {
        const int32_t* v = tri + 3 * ptri[i];
        double A[2] = {vxy[2 * v[0]], vxy[2 * v[0] + 1]};
        double B[2] = {vxy[2 * v[1]], vxy[2 * v[1] + 1]};
        double C[2] = {vxy[2 * v[2]], vxy[2 * v[2] + 1]};
        double xx = txy[2 * pt[i]], xy = txy[2 * pt[i] + 1];
        double m[NB];
        int64_t st = 0, cap = 0;
        if (pkind[i] == 1) self_moments(P, A, B, C, J[ptri[i]], xx, xy, m, &st);
        else near_moments(P, A, B, C, J[ptri[i]], xx, xy, m, &st, &cap);
        moments_to_weights(P, m, J[ptri[i]], xx, xy, A, B, C, pown[i], out + i * P->nq);
        stats[i] = st;
        capped_sum += cap;
    }
    *capped_total = capped_sum;
}

/* Test hook: the panel counts N and M of each fan of a self pair. */
void or_self_panel_counts(const double* A, const double* B, const double* C, double xx, double xy, int32_t* out6) {
    const double* V[3] = {A, B, C};
    for (int e = 0; e < 3; e++) {
        const double* Pp = V[e];
        const double* Qp = V[(e + 1) % 3];
        double dx = Qp[0] - Pp[0], dy = Qp[1] - Pp[1];
        double L = sqrt(dx * dx + dy * dy);
        double st = (dx * (xx - Pp[0]) + dy * (xy - Pp[1])) / L;
        if (st < 0.0) st = 0.0;
        if (st > L) st = L;
        double fxp = Pp[0] + (st / L) * dx, fyp = Pp[1] + (st / L) * dy;
        double delta = sqrt((xx - fxp) * (xx - fxp) + (xy - fyp) * (xy - fyp));
        out6[2 * e] = st > 0.0 ? dyadic_count(st, delta) : -1;
        out6[2 * e + 1] = st < L ? dyadic_count(L - st, delta) : -1;
    }
}

/* Test hook: basis values at points. */
void or_basis(const or_params* P, const double* xi, const double* eta, int64_t n, double* out) {
    for (int64_t i = 0; i < n; i++) basis(P, xi[i], eta[i], out + i * NB);
}

/* Test hook: the raw near / self integrals of the degree <= 4 projection
 * basis (the moments m_a) for a single pair. */
void or_pair_moments(const or_params* P, const double* A, const double* B, const double* C, double J,
                     double xx, double xy, int kind, double* m, int64_t* stat) {
    int64_t cap = 0;
    *stat = 0;
    if (kind == 1) self_moments(P, A, B, C, J, xx, xy, m, stat);
    else near_moments(P, A, B, C, J, xx, xy, m, stat, &cap);
}

/* ================================================================ curved
 * Curved elements (Section 3.1, blending map Eq. for:blend).  A curved
 * element is a counter-clockwise triangle (v0, v1, v2) whose side v0 -> v1
 * is the curve c(xi), xi in [0, 1], c(0) = v0, c(1) = v1; it is given by its
 * deviation from the chord, c(xi) - (1-xi) v0 - xi v1 = xi (1-xi) D(xi), with
 * D(xi) = sum_k a_k T_k(2 xi - 1) (Chebyshev, K+1 coefficients per
 * coordinate).  With gamma(L(1-xi)) = c(xi), gamma(L) = v0, gamma(0) = v1 and
 * the opposite vertex v2, the blending map becomes
 *   rho(xi, eta) = v0 + xi (v1 - v0) + eta (v2 - v0) + xi (1 - xi - eta) D(xi),
 * affine when D = 0.  Near-field lists treat the curved side as its chord
 * (Section 4.1, last remark on curved elements); point location and the
 * preimage of a self target use Newton's method on rho; the near scheme
 * subdivides the reference simplex and maps leaves through rho; the self
 * scheme uses radius-arclength fans in reference coordinates around
 * rho^{-1}(x), with log|rho(y) - x| = log r + log(|rho(y) - x| / r).
 */
typedef struct {
    const double* vxy;
    const int32_t* tri;  /* counter-clockwise */
    const int32_t* cidx; /* per triangle: curve index, -1 straight */
    const double* coef;  /* [ncurve][2][K+1] */
    int K;
} or_geom;

/* D(xi) and dD/dxi */
static void cheb_eval(const double* a, int K, double xi, double* v, double* dv) {
    double t = 2.0 * xi - 1.0;
    double T0 = 1.0, T1 = t, dT0 = 0.0, dT1 = 1.0;
    double s = a[0], ds = 0.0;
    if (K >= 1) { s += a[1] * T1; ds += a[1] * dT1; }
    for (int k = 2; k <= K; k++) {
        double T2 = 2.0 * t * T1 - T0;
        double dT2 = 2.0 * T1 + 2.0 * t * dT1 - dT0;
        s += a[k] * T2;
        ds += a[k] * dT2;
        T0 = T1; T1 = T2; dT0 = dT1; dT1 = dT2;
    }
    *v = s;
    *dv = 2.0 * ds;
}

/* y = rho_T(xi, eta), its Jacobian matrix (columns d/dxi, d/deta) and det */
static void geom_map(const or_geom* g, int64_t T, double xi, double eta, double* y, double* Jm, double* det) {
    const int32_t* v = g->tri + 3 * T;
    double Ax = g->vxy[2 * v[0]], Ay = g->vxy[2 * v[0] + 1];
    double ex = g->vxy[2 * v[1]] - Ax, ey = g->vxy[2 * v[1] + 1] - Ay;
    double fx = g->vxy[2 * v[2]] - Ax, fy = g->vxy[2 * v[2] + 1] - Ay;
    double yx = Ax + (xi * ex + eta * fx), yy = Ay + (xi * ey + eta * fy);
    double a11 = ex, a21 = ey, a12 = fx, a22 = fy;
    int c = g->cidx ? g->cidx[T] : -1;
    if (c >= 0) {
        const double* ax = g->coef + (int64_t)c * 2 * (g->K + 1);
        const double* ay = ax + (g->K + 1);
        double Dx, dDx, Dy, dDy;
        cheb_eval(ax, g->K, xi, &Dx, &dDx);
        cheb_eval(ay, g->K, xi, &Dy, &dDy);
        double b = xi * (1.0 - xi - eta);
        double bx = 1.0 - 2.0 * xi - eta; /* d b / d xi */
        yx += b * Dx;
        yy += b * Dy;
        a11 += bx * Dx + b * dDx;
        a21 += bx * Dy + b * dDy;
        a12 -= xi * Dx; /* d b / d eta = -xi */
        a22 -= xi * Dy;
    }
    y[0] = yx;
    y[1] = yy;
    if (Jm) { Jm[0] = a11; Jm[1] = a21; Jm[2] = a12; Jm[3] = a22; }
    if (det) *det = a11 * a22 - a12 * a21;
}

/* rho_T^{-1}(x) by Newton's method from the chord's affine inverse.
 * Returns the number of iterations, -1 if it did not converge. */
static int geom_inverse(const or_geom* g, int64_t T, double x, double y, double* xi, double* eta) {
    const int32_t* v = g->tri + 3 * T;
    double Ax = g->vxy[2 * v[0]], Ay = g->vxy[2 * v[0] + 1];
    double ex = g->vxy[2 * v[1]] - Ax, ey = g->vxy[2 * v[1] + 1] - Ay;
    double fx = g->vxy[2 * v[2]] - Ax, fy = g->vxy[2 * v[2] + 1] - Ay;
    double J = ex * fy - ey * fx;
    double qx = x - Ax, qy = y - Ay;
    double a = (qx * fy - qy * fx) / J, b = (ex * qy - ey * qx) / J;
    /* quadratic convergence to the rounding level: stop when a step is
     * below 1e-14 or no longer shrinks; fail if it ends above 1e-12 */
    double prev = 1e300;
    for (int it = 0; it < 60; it++) {
        double p[2], M[4], det;
        geom_map(g, T, a, b, p, M, &det);
        double rx = p[0] - x, ry = p[1] - y;
        double da = (M[3] * rx - M[2] * ry) / det, db = (-M[1] * rx + M[0] * ry) / det;
        double step = fabs(da) + fabs(db);
        if (step >= prev && step <= 1e-12 * (1.0 + fabs(a) + fabs(b))) { *xi = a; *eta = b; return it + 1; }
        a -= da;
        b -= db;
        if (step <= 1e-14 * (1.0 + fabs(a) + fabs(b))) { *xi = a; *eta = b; return it + 1; }
        prev = step;
    }
    *xi = a;
    *eta = b;
    return -1;
}

/* Nodes and weights with curved elements (Theorem 3.1 with |J_rho|):
 * y_j = rho_T(xi_k, eta_k), W_j = w_k |det J_rho(xi_k, eta_k)|.  Straight
 * triangles as in or_nodes; curved ones must be given counter-clockwise.
 * J[t] is the chord's 2 * area. */
int or_nodes_curved(const double* vxy, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* cidx,
                    const double* coef, int K, const or_params* P, int32_t* tri_ccw, double* yxy, double* W, double* J) {
    int rc = or_nodes(vxy, nv, tri, nt, P, tri_ccw, yxy, W, J);
    if (rc) return rc;
    or_geom g = {vxy, tri_ccw, cidx, coef, K};
    for (int64_t t = 0; t < nt; t++) {
        if (cidx[t] < 0) continue;
        if (tri_ccw[3 * t + 1] != tri[3 * t + 1]) return -3; /* curved elements must be counter-clockwise */
        for (int k = 0; k < P->nq; k++) {
            int64_t j = t * P->nq + k;
            double det;
            geom_map(&g, t, P->fx[k], P->fy[k], yxy + 2 * j, NULL, &det);
            if (!(det > 0)) return -4;
            W[j] = P->fw[k] * det;
        }
    }
    return 0;
}

/* Point location with curved elements: a straight triangle as in
 * or_locate_one; a curved one holds x when x is on the inner side of its two
 * straight sides and the Newton preimage lies in the reference simplex:
 * eta >= 0 (inner side of the curve), and xi >= -1e-9, xi + eta <= 1 + 1e-9
 * (the straight sides, already decided exactly by the orientation tests; the
 * slack only absorbs the preimage's rounding).  App. A.5 with the polar-angle
 * test replaced by the preimage.  Far from the element the blending map has
 * other roots (its curve term is a polynomial in xi), which lie outside the
 * simplex: the bounds on xi reject them. */
int64_t or_locate_curved_one(const or_geom* g, int64_t nt, double x, double y) {
    for (int64_t t = 0; t < nt; t++) {
        const int32_t* v = g->tri + 3 * t;
        double Ax = g->vxy[2 * v[0]], Ay = g->vxy[2 * v[0] + 1];
        double Bx = g->vxy[2 * v[1]], By = g->vxy[2 * v[1] + 1];
        double Cx = g->vxy[2 * v[2]], Cy = g->vxy[2 * v[2] + 1];
        if (g->cidx[t] < 0) {
            if (orient(Ax, Ay, Bx, By, x, y) >= 0 && orient(Bx, By, Cx, Cy, x, y) >= 0 &&
                orient(Cx, Cy, Ax, Ay, x, y) >= 0)
                return t;
        } else if (orient(Bx, By, Cx, Cy, x, y) >= 0 && orient(Cx, Cy, Ax, Ay, x, y) >= 0) {
            double xi, eta;
            if (geom_inverse(g, t, x, y, &xi, &eta) > 0 && eta >= 0.0 && xi >= -1e-9 && xi + eta <= 1.0 + 1e-9)
                return t;
        }
    }
    return -1;
}

void or_locate_curved(const double* vxy, const int32_t* tri, int64_t nt, const int32_t* cidx, const double* coef,
                      int K, const double* pts, int64_t m, int32_t* out) {
    or_geom g = {vxy, tri, cidx, coef, K};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; i++) out[i] = (int32_t)or_locate_curved_one(&g, nt, pts[2 * i], pts[2 * i + 1]);
}

/* Near scheme on a curved element: the subdivision of Section 3.3 in the
 * reference simplex; the stop test of Section 4.1 on the triangle through
 * the images of the sub-triangle's vertices with J_S = J_T 4^-depth (J_T of
 * the chord); near-rule nodes mapped through rho with weight w_j 4^-depth
 * |det J_rho|. */
static void near_moments_curved(const or_params* P, const or_geom* g, int64_t T, double J, double xx, double xy,
                                double* m, int64_t* leaves, int64_t* capped) {
    subtri stack[4 * 64 + 8];
    int sp = 0;
    stack[sp].v[0] = 0; stack[sp].v[1] = 0; stack[sp].v[2] = 1; stack[sp].v[3] = 0;
    stack[sp].v[4] = 0; stack[sp].v[5] = 1; stack[sp].depth = 0; sp++;
    for (int a = 0; a < NB; a++) m[a] = 0.0;
    while (sp > 0) {
        subtri S = stack[--sp];
        double ph[6];
        for (int i = 0; i < 3; i++) geom_map(g, T, S.v[2 * i], S.v[2 * i + 1], ph + 2 * i, NULL, NULL);
        double JS = ldexp(J, -2 * S.depth);
        int inside = orient(ph[0], ph[1], ph[2], ph[3], xx, xy) >= 0 && orient(ph[2], ph[3], ph[4], ph[5], xx, xy) >= 0 &&
                     orient(ph[4], ph[5], ph[0], ph[1], xx, xy) >= 0;
        int stop = !inside && !tri_near(ph[0], ph[1], ph[2], ph[3], ph[4], ph[5], xx, xy, P->near_degree,
                                        ellipse_R(P->near_what, JS, P->eps, P->near_cn));
        if (!stop && S.depth >= P->depth_cap) { stop = 1; (*capped)++; }
        if (stop) {
            (*leaves)++;
            double sc = ldexp(1.0, -2 * S.depth);
            for (int j = 0; j < P->nn; j++) {
                double xi = S.v[0] + (P->nx[j] * (S.v[2] - S.v[0]) + P->ny[j] * (S.v[4] - S.v[0]));
                double eta = S.v[1] + (P->nx[j] * (S.v[3] - S.v[1]) + P->ny[j] * (S.v[5] - S.v[1]));
                double y[2], det;
                geom_map(g, T, xi, eta, y, NULL, &det);
                double gg = kernelG(xx, xy, y[0], y[1]) * P->nw[j] * sc * det;
                double Kb[NB];
                basis(P, xi, eta, Kb);
                for (int a = 0; a < NB; a++) m[a] += gg * Kb[a];
            }
        } else {
            double m01x = 0.5 * (S.v[0] + S.v[2]), m01y = 0.5 * (S.v[1] + S.v[3]);
            double m12x = 0.5 * (S.v[2] + S.v[4]), m12y = 0.5 * (S.v[3] + S.v[5]);
            double m20x = 0.5 * (S.v[4] + S.v[0]), m20y = 0.5 * (S.v[5] + S.v[1]);
            double ch[4][6] = {{S.v[0], S.v[1], m01x, m01y, m20x, m20y},
                               {m01x, m01y, S.v[2], S.v[3], m12x, m12y},
                               {m20x, m20y, m12x, m12y, S.v[4], S.v[5]},
                               {m12x, m12y, m20x, m20y, m01x, m01y}};
            for (int c = 0; c < 4; c++) {
                memcpy(stack[sp].v, ch[c], sizeof(ch[c]));
                stack[sp].depth = S.depth + 1;
                sp++;
            }
        }
    }
}

/* Self scheme on a curved element (Section 3.4 in reference coordinates):
 * the reference simplex is split at p = rho^{-1}(x) into three fans over its
 * sides; on the fan over side P -> Q (reference length Lr, distance hr from
 * p) the point y(r, s) = p + r (P + s/Lr (Q - P) - p) and
 *   int = int_0^Lr int_0^1 [log r + psi(r, s)] K(y) |det J_rho(y)| r hr dr ds / 2pi,
 *   psi = log(|rho(y) - x| / r)  (smooth; = log r0(s) for straight elements),
 * with the generalized Gaussian rule in r and Gauss-Legendre panels in s
 * graded toward the point of the physical side nearest to x: s~ minimises
 * |rho(side(s)) - x| (Newton on the curved side, projection on the straight
 * ones), delta is that distance, and the panel counts are those of Section
 * 3.4 with the physical chord lengths |F - P|, |Q - F| (F the foot point). */
static double side_dist2(const or_geom* g, int64_t T, const double* Pr, const double* dr, double s, double x, double y,
                         double* F) {
    double yp[2];
    geom_map(g, T, Pr[0] + s * dr[0], Pr[1] + s * dr[1], yp, NULL, NULL);
    if (F) { F[0] = yp[0]; F[1] = yp[1]; }
    return (yp[0] - x) * (yp[0] - x) + (yp[1] - y) * (yp[1] - y);
}

static void self_moments_curved(const or_params* P, const or_geom* g, int64_t T, double xx, double xy, double* m,
                                int64_t* panels) {
    static const double R[3][2] = {{0, 0}, {1, 0}, {0, 1}};
    double pxi, peta;
    geom_inverse(g, T, xx, xy, &pxi, &peta);
    for (int a = 0; a < NB; a++) m[a] = 0.0;
    for (int e = 0; e < 3; e++) {
        const double* Pr = R[e];
        const double* Qr = R[(e + 1) % 3];
        double dr[2] = {Qr[0] - Pr[0], Qr[1] - Pr[1]}; /* side(s) = Pr + s dr, s in [0, 1] */
        double Lr = sqrt(dr[0] * dr[0] + dr[1] * dr[1]);
        double hr = fabs(dr[0] * (peta - Pr[1]) - dr[1] * (pxi - Pr[0])) / Lr;
        if (hr == 0.0) continue;
        double Pp[2], Qp[2];
        geom_map(g, T, Pr[0], Pr[1], Pp, NULL, NULL);
        geom_map(g, T, Qr[0], Qr[1], Qp, NULL, NULL);
        /* foot point: projection on the chord, then Newton on d/ds |side(s) - x|^2 */
        double cx = Qp[0] - Pp[0], cy = Qp[1] - Pp[1];
        double s = ((xx - Pp[0]) * cx + (xy - Pp[1]) * cy) / (cx * cx + cy * cy);
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
        if (e == 0 && g->cidx[T] >= 0) {
            for (int it = 0; it < 30; it++) {
                double h = 1e-6;
                double f0 = side_dist2(g, T, Pr, dr, s, xx, xy, NULL);
                double fp = side_dist2(g, T, Pr, dr, s + h, xx, xy, NULL);
                double fm = side_dist2(g, T, Pr, dr, s - h, xx, xy, NULL);
                double d1 = (fp - fm) / (2 * h), d2 = (fp - 2 * f0 + fm) / (h * h);
                if (!(d2 > 0)) break;
                double step = d1 / d2;
                double sn = s - step;
                if (sn < 0.0) sn = 0.0;
                if (sn > 1.0) sn = 1.0;
                if (fabs(sn - s) < 1e-15) { s = sn; break; }
                s = sn;
            }
        }
        double F[2];
        double delta = sqrt(side_dist2(g, T, Pr, dr, s, xx, xy, F));
        double len0 = sqrt((F[0] - Pp[0]) * (F[0] - Pp[0]) + (F[1] - Pp[1]) * (F[1] - Pp[1]));
        double len1 = sqrt((Qp[0] - F[0]) * (Qp[0] - F[0]) + (Qp[1] - F[1]) * (Qp[1] - F[1]));
        double bnd[2][130];
        int nb[2] = {0, 0};
        if (s > 0.0) {
            int N = dyadic_count(len0, delta);
            bnd[0][nb[0]++] = 0.0;
            for (int i = 1; i <= N; i++) bnd[0][nb[0]++] = (1.0 - ldexp(1.0, -i)) * s;
            bnd[0][nb[0]++] = s;
        }
        if (s < 1.0) {
            int Mm = dyadic_count(len1, delta);
            bnd[1][nb[1]++] = 1.0;
            for (int i = 1; i <= Mm; i++) bnd[1][nb[1]++] = 1.0 - (1.0 - ldexp(1.0, -i)) * (1.0 - s);
            bnd[1][nb[1]++] = s;
        }
        for (int side = 0; side < 2; side++) {
            for (int pi = 0; pi + 1 < nb[side]; pi++) {
                double s0 = bnd[side][pi], s1 = bnd[side][pi + 1];
                (*panels)++;
                for (int l = 0; l < P->nl; l++) {
                    double su = s0 + (s1 - s0) * P->lx[l];   /* parameter in [0, 1] */
                    double ws = fabs((s1 - s0) * P->lw[l]) * Lr; /* reference arc length */
                    double gx = Pr[0] + su * dr[0], gy = Pr[1] + su * dr[1];
                    for (int j = 0; j < P->ng; j++) {
                        double r = P->gr[j];
                        double yxi = pxi + r * (gx - pxi), yeta = peta + r * (gy - peta);
                        double y[2], det;
                        geom_map(g, T, yxi, yeta, y, NULL, &det);
                        double dist = sqrt((y[0] - xx) * (y[0] - xx) + (y[1] - xy) * (y[1] - xy));
                        double lg = log(r) + log(dist / r);
                        double Kb[NB];
                        basis(P, yxi, yeta, Kb);
                        double gg = lg / TWO_PI * ws * hr * P->gw[j] * det;
                        for (int a = 0; a < NB; a++) m[a] += gg * Kb[a];
                    }
                }
            }
        }
    }
}

/* Correction weights with curved elements: straight pairs as or_weights,
 * curved ones with the two schemes above and C_k = w_k sum_a K_a(xi_k) m_a
 * - [k != own] W_k G(x, y_k) with the curved nodes and weights. */
void or_weights_curved(const double* vxy, const int32_t* tri, const double* J, const int32_t* cidx,
                       const double* coef, int K, const or_params* P, const double* yxy, const double* W,
                       const double* txy, const int64_t* pt, const int32_t* ptri, const uint8_t* pkind,
                       const int32_t* pown, int64_t npairs, double* out, int64_t* stats, int64_t* capped_total) {
    or_geom g = {vxy, tri, cidx, coef, K};
    int64_t capped_sum = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : capped_sum)
    for (int64_t i = 0; i < npairs; i++) {
        int64_t T = ptri[i];
        const int32_t* v = tri + 3 * T;
        double A[2] = {vxy[2 * v[0]], vxy[2 * v[0] + 1]};
        double B[2] = {vxy[2 * v[1]], vxy[2 * v[1] + 1]};
        double Cc[2] = {vxy[2 * v[2]], vxy[2 * v[2] + 1]};
        double xx = txy[2 * pt[i]], xy = txy[2 * pt[i] + 1];
        double m[NB];
        int64_t st = 0, cap = 0;
        double* o = out + i * P->nq;
        if (cidx[T] < 0) {
            if (pkind[i] == 1) self_moments(P, A, B, Cc, J[T], xx, xy, m, &st);
            else near_moments(P, A, B, Cc, J[T], xx, xy, m, &st, &cap);
            moments_to_weights(P, m, J[T], xx, xy, A, B, Cc, pown[i], o);
        } else {
            if (pkind[i] == 1) self_moments_curved(P, &g, T, xx, xy, m, &st);
            else near_moments_curved(P, &g, T, J[T], xx, xy, m, &st, &cap);
            for (int k = 0; k < P->nq; k++) {
                double Kb[NB];
                basis(P, P->fx[k], P->fy[k], Kb);
                double s = 0.0;
                for (int a = 0; a < NB; a++) s += Kb[a] * m[a];
                double val = P->fw[k] * s;
                int64_t j = T * P->nq + k;
                if (k != pown[i]) val -= W[j] * kernelG(xx, xy, yxy[2 * j], yxy[2 * j + 1]);
                o[k] = val;
            }
        }
        stats[i] = st;
        capped_sum += cap;
    }
    *capped_total = capped_sum;
}

/* Test hooks: the map, its Jacobian determinant and the Newton preimage. */
void or_map_curved(const double* vxy, const int32_t* tri, const int32_t* cidx, const double* coef, int K,
                   const int64_t* T, const double* xi, const double* eta, int64_t n, double* y, double* det) {
    or_geom g = {vxy, tri, cidx, coef, K};
    for (int64_t i = 0; i < n; i++) geom_map(&g, T[i], xi[i], eta[i], y + 2 * i, NULL, det + i);
}

void or_inverse_curved(const double* vxy, const int32_t* tri, const int32_t* cidx, const double* coef, int K,
                       const int64_t* T, const double* pts, int64_t n, double* ref, int32_t* iters) {
    or_geom g = {vxy, tri, cidx, coef, K};
    for (int64_t i = 0; i < n; i++)
        iters[i] = geom_inverse(&g, T[i], pts[2 * i], pts[2 * i + 1], ref + 2 * i, ref + 2 * i + 1);
}

void or_pair_moments_curved(const or_params* P, const double* vxy, const int32_t* tri, const double* J,
                            const int32_t* cidx, const double* coef, int K, int64_t T, double xx, double xy,
                            int kind, double* m, int64_t* stat) {
    or_geom g = {vxy, tri, cidx, coef, K};
    int64_t cap = 0;
    *stat = 0;
    if (kind == 1) self_moments_curved(P, &g, T, xx, xy, m, stat);
    else near_moments_curved(P, &g, T, J[T], xx, xy, m, stat, &cap);
}
