// Float-float (unevaluated pairs of FP32 values, h + l) arithmetic for the
// correction-weight quadratures.  GB300 runs FP32 at 62x its FP64 rate, so
// the per-node work of the near and self quadratures (Sections 3.3, 3.4) is
// evaluated with error-free transformations in FP32 (about 2^-48 relative
// per operation) instead of FP64; the subdivision tree, its predicates and
// the per-leaf set-up stay FP64.  Every operation is written with explicit
// round-to-nearest intrinsics so the compiler cannot contract or reorder it.
#pragma once
#include <cuda_runtime.h>

struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 f2_from_d(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double f2_to_d(f2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.h, -a.l}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void f2_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// renormalise when |a| >= |b| (or a = 0)
__device__ __forceinline__ f2 f2_fast(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    float s, e;
    f2_two_sum(a.h, b.h, s, e);
    return f2_fast(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 f2_add_f(f2 a, float c) {
    float s, e;
    f2_two_sum(a.h, c, s, e);
    return f2_fast(s, __fadd_rn(e, a.l));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return f2_fast(p, e);
}
// the same product left unnormalised: (p, e) with p = fl(a.h b.h) and
// |e| <= 3 2^-24 |p| (the error of p plus the cross terms), for chains of
// products whose terms are only added (f2_acc1) or multiplied again: the
// cross terms of the next product stay 2^-22 below it, as with a
// normalised pair, and three instructions are saved per product
__device__ __forceinline__ f2 f2_mul_u(f2 a, f2 b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)));
    return {p, e};
}
__device__ __forceinline__ f2 f2_sqr(f2 a) {
    const float p = __fmul_rn(a.h, a.h);
    const float e = __fmaf_rn(__fmul_rn(2.0f, a.h), a.l, __fmaf_rn(a.h, a.h, -p));
    return f2_fast(p, e);
}
// c1 a + c0 for FP32 constants
__device__ __forceinline__ f2 f2_axpb(f2 a, float c1, float c0) {
    const float p = __fmul_rn(c1, a.h);
    const float e = __fmaf_rn(c1, a.l, __fmaf_rn(c1, a.h, -p));
    float s, t;
    f2_two_sum(p, c0, s, t);
    return f2_fast(s, __fadd_rn(t, e));
}
// a 2^k (exact while the parts stay normal)
__device__ __forceinline__ f2 f2_scale(f2 a, float pow2) { return {__fmul_rn(a.h, pow2), __fmul_rn(a.l, pow2)}; }

// acc += g L with the product split exactly (hi) and the cross terms in FP32;
// acc is kept unnormalised (h by two-sum, l gathers the errors).
__device__ __forceinline__ void f2_acc(float& ah, float& al, f2 g, f2 L) {
    const float p = __fmul_rn(g.h, L.h);
    float e = __fmaf_rn(g.h, L.h, -p);
    e = __fmaf_rn(g.h, L.l, __fmaf_rn(g.l, L.h, e));
    float s, t;
    f2_two_sum(ah, p, s, t);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(t, e));
}
__device__ __forceinline__ void f2_acc1(float& ah, float& al, f2 g) {
    float s, t;
    f2_two_sum(ah, g.h, s, t);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(t, g.l));
}

// m += g M_ab(x, y) for the monomial basis M_ab = u^a v^b, u = 3x - 1,
// v = 3y - 1, a + b <= 4, in the order of leg15: the terms g u^a v^b come from
// one chain of 14 products (g u^a, then times v, left unnormalised), each
// added by a two-sum.
__device__ __forceinline__ void f2_mon15_acc_uv(float* mh, float* ml, f2 g, f2 u, f2 v) {
    const f2 t1 = f2_mul_u(g, u), t2 = f2_mul_u(t1, u), t3 = f2_mul_u(t2, u), t4 = f2_mul_u(t3, u);
    const f2 s01 = f2_mul_u(g, v), s02 = f2_mul_u(s01, v), s03 = f2_mul_u(s02, v), s04 = f2_mul_u(s03, v);
    const f2 s11 = f2_mul_u(t1, v), s12 = f2_mul_u(s11, v), s13 = f2_mul_u(s12, v);
    const f2 s21 = f2_mul_u(t2, v), s22 = f2_mul_u(s21, v);
    const f2 s31 = f2_mul_u(t3, v);
    f2_acc1(mh[0], ml[0], g);
    f2_acc1(mh[1], ml[1], t1);
    f2_acc1(mh[2], ml[2], s01);
    f2_acc1(mh[3], ml[3], t2);
    f2_acc1(mh[4], ml[4], s11);
    f2_acc1(mh[5], ml[5], s02);
    f2_acc1(mh[6], ml[6], t3);
    f2_acc1(mh[7], ml[7], s21);
    f2_acc1(mh[8], ml[8], s12);
    f2_acc1(mh[9], ml[9], s03);
    f2_acc1(mh[10], ml[10], t4);
    f2_acc1(mh[11], ml[11], s31);
    f2_acc1(mh[12], ml[12], s22);
    f2_acc1(mh[13], ml[13], s13);
    f2_acc1(mh[14], ml[14], s04);
}
__device__ __forceinline__ void f2_mon15_acc(float* mh, float* ml, f2 g, f2 x, f2 y) {
    f2_mon15_acc_uv(mh, ml, g, f2_axpb(x, 3.0f, -1.0f), f2_axpb(y, 3.0f, -1.0f));
}
// a c for an FP32 constant c (product error kept)
__device__ __forceinline__ f2 f2_mulf(f2 a, float c) {
    const float p = __fmul_rn(c, a.h);
    return f2_fast(p, __fmaf_rn(c, a.l, __fmaf_rn(c, a.h, -p)));
}

// m += g L_ab(x, y) for the tensor-Legendre basis L_ab = P_a(3x - 1) P_b(3y - 1),
// a + b <= 4, in the order of leg15 (n = a + b, then a from n down to 0).
__device__ __forceinline__ void f2_leg15_acc(float* mh, float* ml, f2 g, f2 x, f2 y) {
    const f2 u = f2_axpb(x, 3.0f, -1.0f), v = f2_axpb(y, 3.0f, -1.0f);
    const f2 u2 = f2_sqr(u), v2 = f2_sqr(v);
    const f2 pu2 = f2_axpb(u2, 1.5f, -0.5f), pv2 = f2_axpb(v2, 1.5f, -0.5f);
    const f2 pu3 = f2_mul(u, f2_axpb(u2, 2.5f, -1.5f)), pv3 = f2_mul(v, f2_axpb(v2, 2.5f, -1.5f));
    const f2 pu4 = f2_add_f(f2_mul(u2, f2_axpb(u2, 4.375f, -3.75f)), 0.375f);
    const f2 pv4 = f2_add_f(f2_mul(v2, f2_axpb(v2, 4.375f, -3.75f)), 0.375f);
    f2_acc1(mh[0], ml[0], g);
    f2_acc(mh[1], ml[1], g, u);
    f2_acc(mh[2], ml[2], g, v);
    f2_acc(mh[3], ml[3], g, pu2);
    f2_acc(mh[4], ml[4], g, f2_mul(u, v));
    f2_acc(mh[5], ml[5], g, pv2);
    f2_acc(mh[6], ml[6], g, pu3);
    f2_acc(mh[7], ml[7], g, f2_mul(pu2, v));
    f2_acc(mh[8], ml[8], g, f2_mul(u, pv2));
    f2_acc(mh[9], ml[9], g, pv3);
    f2_acc(mh[10], ml[10], g, pu4);
    f2_acc(mh[11], ml[11], g, f2_mul(pu3, v));
    f2_acc(mh[12], ml[12], g, f2_mul(pu2, pv2));
    f2_acc(mh[13], ml[13], g, f2_mul(u, pv3));
    f2_acc(mh[14], ml[14], g, pv4);
}
