// Far rules (Section 3.2) on the host: the two built-in S3-symmetric rules of
// degree 8 and 9, the tabulated S3-symmetric rules of degree 12-50
// (VP_RULE_SYM(n), vp_tables.h) and generated conical-product rules of any
// total degree n in [VP_RULE_CONICAL_MIN, VP_RULE_CONICAL_MAX], for the order
// sweep of Section 4.2 (raising the far order N_f offloads near-field work to
// the far sum).  A conical-product rule maps the Gauss-Legendre rule of
// m = floor((n + 3)/2) points on [0, 1]^2 to the simplex by
// (u, v) -> (u, (1 - u) v) with Jacobian (1 - u):
//   node k = i m + j:  x = u_i,  y = (1 - u_i) u_j,  w = a_i a_j (1 - u_i),
// exact for total degree 2m - 2 >= n, positive weights, nodes inside.
//
// For every rule the library also needs the weight w-hat of Eq. rho0 and the
// map Q from the P_4 moments of a near pair to its nodal correction weights,
// Q[k][i] = w_k sum_j Hinv[i][j] L_j(x_k, y_k) (the discrete L2 projection
// onto P_4 with the far rule, exact Gram matrix because n >= 8).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstddef>
#include <mutex>
#include <new>
#include <vector>

#include "vp_internal.h"
#include "vp_tables.h"

namespace {

// P_a(t), a <= 4, by Bonnet's recurrence.
long double legendre_ld(int a, long double t) {
    long double p0 = 1.0L, p1 = t;
    if (a == 0) return p0;
    for (int k = 1; k < a; k++) {
        const long double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// Tensor-Legendre basis of P_4 in the device order (total degree n, then a
// from n down to 0): L_ab(x, y) = P_a(3x - 1) P_b(3y - 1).
void leg15_ld(long double x, long double y, long double* L) {
    int i = 0;
    for (int n = 0; n <= 4; n++)
        for (int a = n; a >= 0; a--) L[i++] = legendre_ld(a, 3.0L * x - 1.0L) * legendre_ld(n - a, 3.0L * y - 1.0L);
}

// Gauss-Legendre rule of m points on [0, 1], ascending.  Newton's method on
// P_m(cos theta) in the angle, so that u = sin^2(theta/2) and
// 1 - u = cos^2(theta/2) keep full relative accuracy near both ends.
void gauss01_ld(int m, std::vector<long double>& u, std::vector<long double>& one_minus_u,
                std::vector<long double>& a) {
    const long double pi = 3.141592653589793238462643383279502884L;
    u.assign(m, 0.0L);
    one_minus_u.assign(m, 0.0L);
    a.assign(m, 0.0L);
    for (int i = 0; i < m; i++) {
        long double th = pi * (i + 0.75L) / (m + 0.5L);   // t = cos th descending: u ascending
        long double dp = 0.0L;
        for (int it = 0; it < 100; it++) {
            const long double t = cosl(th);
            long double p0 = 1.0L, p1 = t;
            for (int k = 1; k < m; k++) {
                const long double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
                p0 = p1;
                p1 = p2;
            }
            dp = m * (t * p1 - p0) / (t * t - 1.0L);         // P_m'(t)
            const long double dth = p1 / (dp * sinl(th));    // d P_m(cos th)/d th = -sin th P_m'
            th += dth;
            if (fabsl(dth) < 1e-30L + 4.0L * LDBL_EPSILON * th) {
                if (it > 0) break;
            }
        }
        const long double t = cosl(th), s = sinl(th), h = sinl(0.5L * th), c = cosl(0.5L * th);
        long double p0 = 1.0L, p1 = t;
        for (int k = 1; k < m; k++) {
            const long double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
            p0 = p1;
            p1 = p2;
        }
        dp = m * (t * p1 - p0) / (t * t - 1.0L);
        u[i] = h * h;
        one_minus_u[i] = c * c;
        a[i] = 1.0L / (s * s * dp * dp);                     // 2 / ((1 - t^2) P'^2), halved for [0, 1]
    }
}

struct Rule {
    std::vector<double> x, y, w;
    double what = 0.0;
    int degree = 0;
};

// w-hat of Eq. rho0 for a generated rule: over the three edges, the largest
// weight among the floor((n + 2)/2) nodes nearest the edge, where nodes tied
// with the last of them (distances equal to 1e-9 relative, as the product
// structure makes them in exact arithmetic) are taken too.
double what_ld(const std::vector<long double>& X, const std::vector<long double>& Y,
               const std::vector<long double>& W, int degree) {
    const int n = (int)X.size();
    const int k = std::min(n, (degree + 2) / 2);
    long double best = 0.0L;
    std::vector<long double> d(n), s(n);
    for (int e = 0; e < 3; e++) {
        for (int i = 0; i < n; i++)
            d[i] = e == 0 ? Y[i] : e == 1 ? X[i] : (1.0L - X[i] - Y[i]) * 0.70710678118654752440084436210484903L;
        s = d;
        std::sort(s.begin(), s.end());
        const long double cut = s[k - 1] * (1.0L + 1e-9L);
        for (int i = 0; i < n; i++)
            if (d[i] <= cut) best = std::max(best, W[i]);
    }
    return (double)best;
}

Rule conical_rule(int degree) {
    const int m = (degree + 3) / 2;
    std::vector<long double> u, omu, a;
    gauss01_ld(m, u, omu, a);
    std::vector<long double> X, Y, W;
    Rule r;
    r.degree = degree;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) {
            X.push_back(u[i]);
            Y.push_back(omu[i] * u[j]);
            W.push_back(a[i] * a[j] * omu[i]);
        }
    for (size_t k = 0; k < X.size(); k++) {
        r.x.push_back((double)X[k]);
        r.y.push_back((double)Y[k]);
        r.w.push_back((double)W[k]);
    }
    r.what = what_ld(X, Y, W, degree);
    return r;
}

// Monomial basis M_ab = u^a v^b, u = 3x - 1, v = 3y - 1, in the same order.
void mon15_ld(long double x, long double y, long double* M) {
    int i = 0;
    const long double u = 3.0L * x - 1.0L, v = 3.0L * y - 1.0L;
    for (int n = 0; n <= 4; n++)
        for (int a = n; a >= 0; a--) {
            long double t = 1.0L;
            for (int e = 0; e < a; e++) t *= u;
            for (int e = 0; e < n - a; e++) t *= v;
            M[i++] = t;
        }
}

// Q (tensor-Legendre moments, FP64 kernels) and QM (monomial moments,
// float-float kernels) of a rule.
void projection_q(const Rule& r, std::vector<double>& Q, std::vector<double>& QM) {
    const int nq = (int)r.w.size();
    Q.assign((size_t)nq * VP_NB, 0.0);
    QM.assign((size_t)nq * VP_NB, 0.0);
    for (int k = 0; k < nq; k++) {
        long double L[VP_NB], M[VP_NB];
        leg15_ld(r.x[k], r.y[k], L);
        mon15_ld(r.x[k], r.y[k], M);
        for (int i = 0; i < VP_NB; i++) {
            long double s = 0.0L, sm = 0.0L;
            for (int j = 0; j < VP_NB; j++) {
                s += (long double)VP_LEG15_HINV[i * VP_NB + j] * L[j];
                sm += (long double)VP_MON15_HINV[i * VP_NB + j] * M[j];
            }
            Q[(size_t)k * VP_NB + i] = (double)((long double)r.w[k] * s);
            QM[(size_t)k * VP_NB + i] = (double)((long double)r.w[k] * sm);
        }
    }
}

}  // namespace

void root_leaf_map(const double* QM, int nq, float2* B2) {
    for (int j = 0; j < VP_NNEAR; j++) {
        long double M[VP_NB];
        mon15_ld(VP_NEAR33_X[j], VP_NEAR33_Y[j], M);
        for (int k = 0; k < nq; k++) {
            long double b = 0.0L;
            for (int i = 0; i < VP_NB; i++) b += (long double)QM[(size_t)k * VP_NB + i] * M[i];
            const double bd = (double)b;
            const float h = (float)bd;
            B2[(size_t)j * nq + k] = make_float2(h, (float)(bd - (double)h));
        }
    }
}

namespace {

bool conical_code(int32_t rule) {
    return rule >= VP_RULE_CONICAL(VP_RULE_CONICAL_MIN) && rule <= VP_RULE_CONICAL(VP_RULE_CONICAL_MAX);
}

// The tabulated S3-symmetric rule of VP_RULE_SYM(n), or null.
const VpSymRule* sym_entry(int32_t rule) {
    for (const VpSymRule& r : VP_SYM_RULES)
        if (rule == VP_RULE_SYM(r.degree)) return &r;
    return nullptr;
}

Rule sym_rule(const VpSymRule& t) {
    Rule r;
    r.degree = t.degree;
    r.x.assign(t.x, t.x + t.n);
    r.y.assign(t.y, t.y + t.n);
    r.w.assign(t.w, t.w + t.n);
    r.what = t.what;
    return r;
}

// A generated (conical) or tabulated (symmetric) far rule.
Rule host_rule(int32_t rule) {
    if (const VpSymRule* t = sym_entry(rule)) return sym_rule(*t);
    return conical_rule(rule - VP_RULE_CONICAL(0));
}

}  // namespace

bool far_rule_valid(int32_t rule) {
    return rule == VP_RULE_16_D8 || rule == VP_RULE_19_D9 || conical_code(rule) || sym_entry(rule);
}

int far_rule_nq(int32_t rule) {
    if (rule == VP_RULE_16_D8 || rule == VP_RULE_19_D9) return rule;
    if (const VpSymRule* t = sym_entry(rule)) return t->n;
    if (!conical_code(rule)) return 0;
    const int m = (rule - VP_RULE_CONICAL(0) + 3) / 2;
    return m * m;
}

int far_rule_get(vp_ctx* ctx, int32_t rule, FarRule* out) {
    if (rule == VP_RULE_16_D8 || rule == VP_RULE_19_D9) {
        const int ri = rule == VP_RULE_16_D8 ? 0 : 1;
        const char* base = (const char*)ctx->d_tables;
        const VpTables& t = ctx->h_tables;
        FarRule r;
        r.code = rule;
        r.degree = t.far_degree[ri];
        r.what = t.far_what[ri];
        r.builtin = ri;
        r.dev.nq = t.nq[ri];
        r.dev.x = (const double*)(base + offsetof(VpTables, fx) + ri * sizeof(t.fx[0]));
        r.dev.y = (const double*)(base + offsetof(VpTables, fy) + ri * sizeof(t.fy[0]));
        r.dev.w = (const double*)(base + offsetof(VpTables, fw) + ri * sizeof(t.fw[0]));
        r.dev.Q = (const double*)(base + offsetof(VpTables, Q) + ri * sizeof(t.Q[0]));
        r.dev.Q2 = (const float2*)(base + offsetof(VpTables, Q2) + ri * sizeof(t.Q2[0]));
        r.dev.B2 = (const float2*)(base + offsetof(VpTables, B2) + ri * sizeof(t.B2[0]));
        *out = r;
        return VP_OK;
    }
    if (!conical_code(rule) && !sym_entry(rule)) return vp_set_error(ctx, VP_ERR_INVALID_ARG, "unknown far rule");
    std::lock_guard<std::mutex> lk(ctx->rule_mu);
    for (const FarRule& r : ctx->gen_rules)
        if (r.code == rule) {
            *out = r;
            return VP_OK;
        }
    const Rule g = host_rule(rule);
    const int nq = (int)g.w.size();
    std::vector<double> Q, QM;
    projection_q(g, Q, QM);
    const size_t nd = (size_t)nq * (3 + VP_NB);
    std::vector<char> blob(nd * sizeof(double) + (size_t)nq * (VP_NB + VP_NNEAR) * sizeof(float2));
    double* hd = (double*)blob.data();
    std::copy(g.x.begin(), g.x.end(), hd);
    std::copy(g.y.begin(), g.y.end(), hd + nq);
    std::copy(g.w.begin(), g.w.end(), hd + 2 * nq);
    std::copy(Q.begin(), Q.end(), hd + 3 * nq);
    float2* hq2 = (float2*)(blob.data() + nd * sizeof(double));
    for (size_t i = 0; i < QM.size(); i++) {
        const float h = (float)QM[i];
        hq2[i] = make_float2(h, (float)(QM[i] - (double)h));
    }
    root_leaf_map(QM.data(), nq, hq2 + (size_t)nq * VP_NB);
    FarRule r;
    r.code = rule;
    r.degree = g.degree;
    r.what = g.what;
    r.builtin = -1;
    if (cudaMalloc(&r.d_buf, blob.size()) != cudaSuccess)
        return vp_set_error(ctx, VP_ERR_OOM, "far rule: device allocation failed");
    if (cudaMemcpy(r.d_buf, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(r.d_buf);
        return vp_set_error(ctx, VP_ERR_CUDA, "far rule: copy failed");
    }
    const double* dd = (const double*)r.d_buf;
    r.dev.nq = nq;
    r.dev.x = dd;
    r.dev.y = dd + nq;
    r.dev.w = dd + 2 * nq;
    r.dev.Q = dd + 3 * nq;
    r.dev.Q2 = (const float2*)((const char*)r.d_buf + nd * sizeof(double));
    r.dev.B2 = r.dev.Q2 + (size_t)nq * VP_NB;
    ctx->gen_rules.push_back(r);
    *out = r;
    return VP_OK;
}

void far_rules_free(vp_ctx* ctx) {
    for (FarRule& r : ctx->gen_rules)
        if (r.d_buf) cudaFree(r.d_buf);
    ctx->gen_rules.clear();
}

extern "C" int vp_far_rule(int32_t rule, double* x, double* y, double* w, double* what, int32_t* degree,
                           int32_t cap, int32_t* n) {
    if (!far_rule_valid(rule)) return VP_ERR_INVALID_ARG;
    Rule g;
    if (rule == VP_RULE_16_D8 || rule == VP_RULE_19_D9) {
        const bool r16 = rule == VP_RULE_16_D8;
        const int nq = rule;
        g.x.assign(r16 ? VP_FAR16_X : VP_FAR19_X, (r16 ? VP_FAR16_X : VP_FAR19_X) + nq);
        g.y.assign(r16 ? VP_FAR16_Y : VP_FAR19_Y, (r16 ? VP_FAR16_Y : VP_FAR19_Y) + nq);
        g.w.assign(r16 ? VP_FAR16_W : VP_FAR19_W, (r16 ? VP_FAR16_W : VP_FAR19_W) + nq);
        g.what = r16 ? VP_FAR16_WHAT : VP_FAR19_WHAT;
        g.degree = r16 ? VP_FAR16_DEGREE : VP_FAR19_DEGREE;
    } else {
        g = host_rule(rule);
    }
    const int32_t len = (int32_t)g.w.size();
    if (n) *n = len;
    if (what) *what = g.what;
    if (degree) *degree = g.degree;
    if (cap < len) return (x || y || w) ? VP_ERR_INVALID_ARG : VP_OK;
    for (int32_t i = 0; i < len; i++) {
        if (x) x[i] = g.x[i];
        if (y) y[i] = g.y[i];
        if (w) w[i] = g.w[i];
    }
    return VP_OK;
}
