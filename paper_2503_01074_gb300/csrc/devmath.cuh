// Device helpers shared by the ray cast, the DVL and the sonar post-processing:
// float3 arithmetic, float-float arithmetic (error-free transforms) and the
// certified FP32 / exact float-float Moller-Trumbore tests.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sonar_internal.cuh"

namespace sonar {
namespace {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float l1(float3 a) { return fabsf(a.x) + fabsf(a.y) + fabsf(a.z); }

// ---- float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2 ----
// Error-free transforms (Knuth's two-sum, FMA-based two-product) carried out
// with explicit round-to-nearest operations so that no contraction or
// reassociation can change them.  About 48 significand bits, all on the FP32
// pipes.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff ff_quick(float a, float b) {   // requires |a| >= |b|
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s = ff_quick(s.hi, __fadd_rn(s.lo, t.hi));
    return ff_quick(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_quick(p, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
    return ff_quick(p, e);
}
__device__ __forceinline__ int ff_sign(ff a) {
    return a.hi > 0.0f ? 1 : a.hi < 0.0f ? -1 : (a.lo > 0.0f ? 1 : a.lo < 0.0f ? -1 : 0);
}
__device__ __forceinline__ ff ff_dot(const ff a[3], const ff b[3]) {
    return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

// ---------------------------------------------------------------------------
// ray / triangle
// ---------------------------------------------------------------------------

// FP32 Moller-Trumbore with a certified error bound.  Returns 0 for a certain
// miss, 1 for a certain hit (t set), 2 when FP32 cannot decide.  Each bound is
// g * (product of the magnitudes entering the numerator) / |det|, with
// g = 2^-19 (32 unit roundoffs), which covers the rounding of the edge vectors,
// of the FP32 direction against the exact one, and of the cross and dot
// products.
__device__ __forceinline__ int mt32(float3 o, float3 d, float4 a, float4 b, float4 c, float& t) {
    const float3 v0 = f3(a.x, a.y, a.z);
    const float3 e1 = sub(f3(b.x, b.y, b.z), v0), e2 = sub(f3(c.x, c.y, c.z), v0);
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    const float3 s = sub(o, v0);
    const float3 q = cross3(s, e1);
    const float un = dot3(s, p), vn = dot3(d, q), tn = dot3(e2, q);
    const float g = 0x1p-19f;
    const float ad = l1(d), as = l1(s), ae1 = l1(e1), ae2 = l1(e2);
    const float Edet = g * ae1 * ad * ae2;
    const float adet = fabsf(det);
    if (adet <= Edet) return 2;   // near-parallel: decided exactly
    const float inv = 1.0f / det;
    const float u = un * inv, v = vn * inv, w = 1.0f - u - v;
    t = tn * inv;
    const float ia = fabsf(inv);   // = 1 / |det| exactly (the rounding of 1/x is odd in x)
    const float eu = (g * as * ad * ae2 + fabsf(u) * Edet) * ia;
    const float ev = (g * ad * as * ae1 + fabsf(v) * Edet) * ia;
    const float ew = eu + ev + 0x1p-22f;
    const float et = (g * ae2 * as * ae1 + fabsf(t) * Edet) * ia;
    if (u < -eu || v < -ev || w < -ew || t < -et) return 0;
    if (u > eu && v > ev && w > ew && t > et) return 1;
    return 2;
}

// Moller-Trumbore on the exact ray in float-float, without division: with
// D = |det| and U, V, T the u, v, t numerators times sign(det), the test
// "det != 0, u >= 0, v >= 0, u + v <= 1, t > 0" becomes
// "D != 0, U >= 0, V >= 0, D - U - V >= 0, T > 0"; t = T / D along w.
// Edge vectors and s = o - v0 are exact (two-sum of FP32 inputs).
__device__ __forceinline__ bool mt_ff(const float o[3], const ff d[3], float4 a, float4 b, float4 c, ff& D,
                                      ff& T) {
    const ff e1[3] = {ff_two_sum(b.x, -a.x), ff_two_sum(b.y, -a.y), ff_two_sum(b.z, -a.z)};
    const ff e2[3] = {ff_two_sum(c.x, -a.x), ff_two_sum(c.y, -a.y), ff_two_sum(c.z, -a.z)};
    const ff sv[3] = {ff_two_sum(o[0], -a.x), ff_two_sum(o[1], -a.y), ff_two_sum(o[2], -a.z)};
    const ff p[3] = {ff_sub(ff_mul(d[1], e2[2]), ff_mul(d[2], e2[1])),
                     ff_sub(ff_mul(d[2], e2[0]), ff_mul(d[0], e2[2])),
                     ff_sub(ff_mul(d[0], e2[1]), ff_mul(d[1], e2[0]))};
    const ff det = ff_dot(e1, p);
    const int sg = ff_sign(det);
    if (sg == 0) return false;
    ff u = ff_dot(sv, p);
    const ff q[3] = {ff_sub(ff_mul(sv[1], e1[2]), ff_mul(sv[2], e1[1])),
                     ff_sub(ff_mul(sv[2], e1[0]), ff_mul(sv[0], e1[2])),
                     ff_sub(ff_mul(sv[0], e1[1]), ff_mul(sv[1], e1[0]))};
    ff v = ff_dot(d, q);
    ff t = ff_dot(e2, q);
    D = det;
    if (sg < 0) { D = ff_neg(det); u = ff_neg(u); v = ff_neg(v); t = ff_neg(t); }
    if (ff_sign(u) < 0 || ff_sign(v) < 0 || ff_sign(ff_sub(ff_sub(D, u), v)) < 0 || ff_sign(t) <= 0) return false;
    T = t;
    return true;
}


// Exact uint -> float for v < 2^23 without a conversion instruction.
__device__ __forceinline__ float small_u2f(uint32_t v) {
    return __uint_as_float(0x4B000000u | v) - 8388608.0f;
}

}  // namespace
}  // namespace sonar
