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
#define MAXQ 64

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
