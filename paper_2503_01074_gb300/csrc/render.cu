// Sonar rendering kernels (OceanSim, arXiv 2503.01074, Sec. III-A-2).
//
// k_trace             one ray per thread, warps on compact beam x elevation
//                     patches: ray generation -> closest hit (LBVH walk,
//                     Moller-Trumbore) -> range/azimuth bin -> 16-byte hit record.
// k_bin               one work unit = whole azimuth columns of one sensor: the
//                     units' hit records -> intensity (Eq. 2, two-way) -> polar
//                     binning into a shared-memory column block -> Eq. 3-6 noise
//                     per bin -> I~ to HBM.  A unit owns its columns, so every
//                     polar bin is written exactly once: no global atomics, no
//                     memset of the image.
// k_norm_rows         range-wise normalisation: one warp per range row takes the
//                     row maximum of I~ and writes N = I~ / max.
// k_fan_tiles         fan resample of the normalised image, tiles of pixels.
// adjoint             per-group (row) Jacobian terms, then a per-ray gather of
//                     dL/dP into (dalpha, dgain, dmu) over ray chunks, and a
//                     fixed-order final reduction (deterministic).
//
// Ray casting precision: the walk and the triangle tests run in FP32.  A test
// whose barycentric or distance outcome lies inside a certified FP32 error
// bound, and any two candidates within 2e-5 t of each other, are re-decided
// exactly in float-float arithmetic (about 48 significant bits, on the FP32
// pipes) against the exact ray, whose direction comes from per-sensor sin/cos
// tables computed in FP64 once; hit decisions therefore agree with an FP64
// reference except for genuinely ambiguous rays.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "sonar_host.h"
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

// ---------------------------------------------------------------------------
// rays
// ---------------------------------------------------------------------------

__device__ __forceinline__ float3 ray_dir32(const SensorDev& s, int i, int j) {
    const float phi = fmaf((float)i + 0.5f, s.hfov / (float)s.nb, -0.5f * s.hfov);
    const float th = fmaf((float)j + 0.5f, s.vfov / (float)s.ne, -0.5f * s.vfov);
    float sp, cp, st, ct;
    sincosf(phi, &sp, &cp);
    sincosf(th, &st, &ct);
    const float dx = sp * ct, dy = cp * ct, dz = st;
    const float3 w = f3(fmaf(s.rot[0], dx, fmaf(s.rot[1], dy, s.rot[2] * dz)),
                        fmaf(s.rot[3], dx, fmaf(s.rot[4], dy, s.rot[5] * dz)),
                        fmaf(s.rot[6], dx, fmaf(s.rot[7], dy, s.rot[8] * dz)));
    const float inv = 1.0f / sqrtf(dot3(w, w));
    return f3(w.x * inv, w.y * inv, w.z * inv);
}

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

// The exact ray of (i, j) in float-float, unnormalised: w = R ds with ds from
// the sensor's float-float sine/cosine tables (beam i, elevation j).  The hit
// decisions below only use signs and ratios, which a positive scale leaves
// unchanged.
__device__ __forceinline__ void ray_dir_ff(const SensorDev& s, int i, int j, ff w[3]) {
    const float4 bp = __ldg(s.trig + i), el = __ldg(s.trig + s.nb + j);
    const ff sp{bp.x, bp.y}, cp{bp.z, bp.w}, st{el.x, el.y}, ct{el.z, el.w};
    const ff ds[3] = {ff_mul(sp, ct), ff_mul(cp, ct), st};
    for (int a = 0; a < 3; ++a)
        w[a] = ff_add(ff_add(ff_mulf(ds[0], s.rot[3 * a]), ff_mulf(ds[1], s.rot[3 * a + 1])),
                      ff_mulf(ds[2], s.rot[3 * a + 2]));
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
    const float ia = 1.0f / adet;
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

// ---------------------------------------------------------------------------
// closest hit: LBVH walk with a short stack
// ---------------------------------------------------------------------------

// The exact decisions, out of line (rarely needed; they would otherwise add
// registers to the FP32 walk) and in float-float on the FP32 pipes.
//
// exact_hit: does the exact ray of (i, j) hit the triangle?  *t = the hit
// distance in FP32.
__device__ __noinline__ bool exact_hit(const SensorDev& s, int i, int j, float4 a, float4 b, float4 c, float* t) {
    ff w[3];
    ray_dir_ff(s, i, j, w);
    const float o[3] = {s.pos[0], s.pos[1], s.pos[2]};
    ff D, T;
    if (!mt_ff(o, w, a, b, c, D, T)) return false;
    const float len = sqrtf(w[0].hi * w[0].hi + w[1].hi * w[1].hi + w[2].hi * w[2].hi);
    *t = (T.hi / D.hi) * len;
    return true;
}

// exact_closer: along the exact ray of (i, j), is triangle `p` (index id_p) the
// closest-hit choice over triangle `q` (index id_q)?  Nearer exact distance
// first (T_p / D_p < T_q / D_q, compared as T_p D_q < T_q D_p), then the lower
// index; a triangle the exact ray misses never wins.
__device__ __noinline__ bool exact_closer(const SensorDev& s, int i, int j, const float4* p, uint32_t id_p,
                                          const float4* q, uint32_t id_q) {
    ff w[3];
    ray_dir_ff(s, i, j, w);
    const float o[3] = {s.pos[0], s.pos[1], s.pos[2]};
    ff Dp, Tp, Dq, Tq;
    if (!mt_ff(o, w, __ldg(p), __ldg(p + 1), __ldg(p + 2), Dp, Tp)) return false;
    if (!mt_ff(o, w, __ldg(q), __ldg(q + 1), __ldg(q + 2), Dq, Tq)) return true;
    const int c = ff_sign(ff_sub(ff_mul(Tp, Dq), ff_mul(Tq, Dp)));
    return c < 0 || (c == 0 && id_p < id_q);
}

// Float-float sine and cosine tables of the sensor's beam azimuths
// phi_i = -H/2 + (i + 1/2) H / N_b and elevations theta_j = -V/2 + (j + 1/2) V / N_e
// (computed in FP64 once per sensor, split into hi + lo floats): trig[i] for
// beams, trig[N_b + j] for elevations, each (sin hi, sin lo, cos hi, cos lo).
__global__ void k_trig(const SensorDev* sensors, SensorDev one) {
    const SensorDev& s = sensors ? sensors[blockIdx.y] : one;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.nb + s.ne) return;
    double a;
    if (k < s.nb) {
        const double H = s.hfov;
        a = -H / 2.0 + (k + 0.5) * H / s.nb;
    } else {
        const double V = s.vfov;
        a = -V / 2.0 + (k - s.nb + 0.5) * V / s.ne;
    }
    double sn, cs;
    sincos(a, &sn, &cs);
    const float sh = (float)sn, ch = (float)cs;
    s.trig[k] = make_float4(sh, (float)(sn - (double)sh), ch, (float)(cs - (double)ch));
}

// Range bin of a hit, or -1 when r is outside [r_min, r_max).
__device__ __forceinline__ int range_bin(const SensorDev& s, float r) {
    if (!(r >= s.rmin && r < s.rmax)) return -1;
    const int br = (int)floorf((r - s.rmin) * s.inv_dr);
    return br < s.nr - 1 ? br : s.nr - 1;
}

// Azimuth bin of beam i: floor((2i + 1) naz / (2 nb)), in 32-bit integers when
// the product fits (it does whenever nb * naz < 2^30).
__device__ __forceinline__ int az_bin(const SensorDev& s, int i) {
    if ((int64_t)s.nb * s.naz < (1ll << 30)) return (int)(((2u * i + 1u) * (uint32_t)s.naz) / (2u * (uint32_t)s.nb));
    return (int)(((2ll * i + 1) * s.naz) / (2ll * s.nb));
}

// Exact uint -> float for v < 2^23 without a conversion instruction.
__device__ __forceinline__ float small_u2f(uint32_t v) {
    return __uint_as_float(0x4B000000u | v) - 8388608.0f;
}

// ---------------------------------------------------------------------------
// trace: one ray per thread, hit record out
// ---------------------------------------------------------------------------

// Each block is one warp on a tile of tb beams x (32 / tb) elevations of one
// sensor: lane l traces beam i0 + l % tb, elevation j0 + l / tb, so that the
// warp's rays sample a compact patch of the field of view.  (One-warp blocks
// free their slot as soon as their rays are done.)  Records go to their
// canonical index i * n_elev + j.
//
// The walk over the 4-wide hierarchy is a while-while loop: a lane descends
// nearest child first, pushing the other entered children; a lane that
// reaches a leaf parks it and keeps descending until every active lane of the
// warp holds one, so that the triangle tests run together.  A lane whose ray
// is finished writes its record at once and idles until the warp is done.
// With STATS the kernel also counts node visits and triangle tests and marks
// the nodes and triangles it touches (records are then not written).
template <int MINB, bool STATS>
__global__ void __launch_bounds__(32, MINB) k_trace(TraceArgs a) {
    __shared__ SensorDev S;
    __shared__ SceneDev SC;
    __shared__ int s_tile;
    if (threadIdx.x == 0) {
        if (a.sensors) {
            const int2 m = a.block_map[blockIdx.x];
            S = a.sensors[m.x];
            SC = a.scenes[S.scene];
            s_tile = m.y;
        } else {
            S = a.one;
            SC = a.one_scene;
            s_tile = blockIdx.x;
        }
    }
    __syncthreads();
    const int tb = S.tb, te = 32 / S.tb;
    const int tiles_b = (S.nb + tb - 1) / tb;
    const int ty = s_tile / tiles_b, tx = s_tile - ty * tiles_b;
    const int lane = threadIdx.x;
    const int ri = tx * tb + (lane % tb);
    const int rj = ty * te + lane / tb;
    const SceneDev& sc = SC;
    const sonar_params& p = a.params;
    const float tlimit = p.clip_tmax ? S.rmax : CUDART_INF_F;
    const float3 o = f3(S.pos[0], S.pos[1], S.pos[2]);
    const bool inside = ri < S.nb && rj < S.ne;
    const float3 d = inside ? ray_dir32(S, ri, rj) : f3(0.0f, 0.0f, 1.0f);
    const float tiny = 1e-20f;
    const float3 inv = f3(1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                          1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                          1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    const float3 oinv = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    int32_t stack[kStackMax];
    int sp = 0, best = -1;
    uint32_t best_id = 0xFFFFFFFFu;
    float best_t = tlimit;
    uint64_t visits = 0, tests = 0, exact_n = 0;
    // `node`: the internal node to visit next (or kEmpty); `leaf`: a parked
    // leaf whose triangles wait to be tested (0 = none; leaf handles are negative)
    int32_t node = inside ? sc.root : kEmpty, leaf = 0;
    if (node < 0 && node != kEmpty) { leaf = node; node = kEmpty; }
    bool live = inside;
    for (;;) {
        if (live) {
            while (node >= 0) {
                const float4* pn = sc.nodes + 8 * (int64_t)node;
                const float4 lx = __ldg(pn), hx = __ldg(pn + 1), ly = __ldg(pn + 2), hy = __ldg(pn + 3);
                const float4 lz = __ldg(pn + 4), hz = __ldg(pn + 5);
                const int4 ch = __ldg(reinterpret_cast<const int4*>(pn + 6));
                if (STATS) {
                    ++visits;
                    atomicOr(a.tc.node_bits + (node >> 5), 1u << (node & 31));
                }
                const float tcut = best_t * 1.00002f;
                const float lxs[4] = {lx.x, lx.y, lx.z, lx.w}, hxs[4] = {hx.x, hx.y, hx.z, hx.w};
                const float lys[4] = {ly.x, ly.y, ly.z, ly.w}, hys[4] = {hy.x, hy.y, hy.z, hy.w};
                const float lzs[4] = {lz.x, lz.y, lz.z, lz.w}, hzs[4] = {hz.x, hz.y, hz.z, hz.w};
                const int32_t hs[4] = {ch.x, ch.y, ch.z, ch.w};
                // sort key per child: entry distance bits (>= 0, so integer order
                // is distance order) with the child slot in the two low bits; a
                // missed child sorts last as 0xFFFFFFFF
                uint32_t key[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float t0 = fmaf(lxs[c], inv.x, -oinv.x), t1 = fmaf(hxs[c], inv.x, -oinv.x);
                    float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
                    t0 = fmaf(lys[c], inv.y, -oinv.y); t1 = fmaf(hys[c], inv.y, -oinv.y);
                    lo = fmaxf(lo, fminf(t0, t1)); hi = fminf(hi, fmaxf(t0, t1));
                    t0 = fmaf(lzs[c], inv.z, -oinv.z); t1 = fmaf(hzs[c], inv.z, -oinv.z);
                    lo = fmaxf(fmaxf(lo, fminf(t0, t1)), 0.0f); hi = fminf(fminf(hi, fmaxf(t0, t1)), tcut);
                    const bool hit = hs[c] != kEmpty && lo <= hi * 1.0000005f;
                    key[c] = hit ? ((__float_as_uint(lo) & ~3u) | (uint32_t)c) : 0xFFFFFFFFu;
                }
#define SONAR_USORT(x, y)                                    \
                {                                            \
                    const uint32_t mn = min(key[x], key[y]); \
                    key[y] = max(key[x], key[y]);            \
                    key[x] = mn;                             \
                }
                SONAR_USORT(0, 1) SONAR_USORT(2, 3) SONAR_USORT(0, 2) SONAR_USORT(1, 3) SONAR_USORT(1, 2)
#undef SONAR_USORT
                const int nhit = (key[0] != 0xFFFFFFFFu) + (key[1] != 0xFFFFFFFFu) + (key[2] != 0xFFFFFFFFu) +
                                 (key[3] != 0xFFFFFFFFu);
                if (nhit == 0) {
                    node = sp > 0 ? stack[--sp] : kEmpty;
                } else {
                    if (sp + nhit - 1 > kStackMax) {   // cannot happen for a checked height: give up the ray
                        atomicOr(a.err, SONAR_DEVERR_STACK);
                        node = kEmpty;
                        leaf = 0;
                        sp = 0;
                        best = -1;
                        break;
                    }
#pragma unroll
                    for (int c = 3; c >= 1; --c) {
                        if (c < nhit) {
                            const uint32_t k = key[c] & 3u;
                            stack[sp++] = k == 0 ? hs[0] : k == 1 ? hs[1] : k == 2 ? hs[2] : hs[3];
                        }
                    }
                    const uint32_t k = key[0] & 3u;
                    node = k == 0 ? hs[0] : k == 1 ? hs[1] : k == 2 ? hs[2] : hs[3];
                }
                if (node < 0 && node != kEmpty && leaf == 0) {   // park the leaf, keep descending
                    leaf = node;
                    node = sp > 0 ? stack[--sp] : kEmpty;
                }
                if (!__any_sync(__activemask(), leaf == 0)) break;
            }
            while (leaf != 0) {
                // a run of triangles in leaf order
                const int32_t x = ~leaf;
                const int32_t first = x >> 3, count = (x & 7) + 1;
                for (int k = 0; k < count; ++k) {
                    const int32_t f = first + k;
                    if (f >= sc.n_tris) {
                        atomicOr(a.err, SONAR_DEVERR_INDEX);
                        break;
                    }
                    const float4* tp = sc.tris + 3 * (int64_t)f;
                    const float4 va = __ldg(tp), vb = __ldg(tp + 1), vc = __ldg(tp + 2);
                    if (STATS) {
                        ++tests;
                        atomicOr(a.tc.tri_bits + (f >> 5), 1u << (f & 31));
                    }
                    float t;
                    const int r = mt32(o, d, va, vb, vc, t);
                    if (r == 0) continue;
                    if (r == 2) {
                        if (STATS) ++exact_n;
                        if (!exact_hit(S, ri, rj, va, vb, vc, &t)) continue;
                    }
                    if (!(t < tlimit)) continue;
                    const uint32_t id = __float_as_uint(vb.w);
                    bool take;
                    if (best < 0) {
                        take = true;
                    } else if (fabsf(t - best_t) <= 2e-5f * fmaxf(t, best_t)) {
                        // near tie: decide on the exact distances, then on the caller's index
                        if (STATS) ++exact_n;
                        take = exact_closer(S, ri, rj, tp, id, sc.tris + 3 * (int64_t)best, best_id);
                    } else {
                        take = t < best_t;
                    }
                    if (take) {
                        best = f;
                        best_id = id;
                        best_t = t;
                    }
                }
                leaf = 0;
                if (node < 0 && node != kEmpty) {   // the next stacked entry is a leaf too
                    leaf = node;
                    node = sp > 0 ? stack[--sp] : kEmpty;
                }
            }
        }
        if (live && node == kEmpty) {
            // the ray is finished: its hit record (bin key, triangle, range, incidence)
            live = false;
            if (!STATS) {
                uint32_t key = kNoKey, orig = 0xFFFFFFFFu, cosb = 0u;
                float tr = CUDART_INF_F;
                if (best >= 0) {
                    const float4* tp = sc.tris + 3 * (int64_t)best;
                    const float4 va = __ldg(tp), vb = __ldg(tp + 1), vc = __ldg(tp + 2);
                    const float3 v0 = f3(va.x, va.y, va.z);
                    const float3 n = cross3(sub(f3(vb.x, vb.y, vb.z), v0), sub(f3(vc.x, vc.y, vc.z), v0));
                    const float dn = dot3(d, n) / sqrtf(dot3(n, n));
                    orig = __float_as_uint(vb.w);
                    tr = best_t;
                    cosb = __float_as_uint(p.two_sided ? fabsf(dn) : fmaxf(-dn, 0.0f));
                    const int br = range_bin(S, best_t);
                    if (br >= 0) key = (uint32_t)(br * S.naz + az_bin(S, ri));
                }
                *reinterpret_cast<uint4*>(a.hits + S.hits_off + (int64_t)ri * S.ne + rj) =
                    make_uint4(key, orig, __float_as_uint(tr), cosb);
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, live) == 0u) break;
    }
    if (STATS) {
        atomicAdd(a.tc.visits, (unsigned long long)visits);
        atomicAdd(a.tc.tests, (unsigned long long)tests);
        atomicAdd(a.tc.exact, (unsigned long long)exact_n);
    }
}

// ---------------------------------------------------------------------------
// bin + noise: one work unit = whole azimuth columns of one sensor
// ---------------------------------------------------------------------------

__device__ __forceinline__ void load_unit(const BinArgs& a, int u, SensorDev* S, SceneDev* SC, Unit* U) {
    if (a.units) {
        *U = a.units[u];
        *S = a.sensors[U->sensor];
        *SC = a.scenes[S->scene];
    } else {
        *S = a.one;
        *SC = a.one_scene;
        U->sensor = 0;
        U->c0 = u * a.one.cols;
        U->c1 = min(U->c0 + a.one.cols, a.one.naz);
        U->rays = 0;
    }
}

// The unit's rays are the contiguous hit records of its beams.  Their scores
// s = mu[m] cos exp(-2 alpha r) gain are summed into a shared-memory column
// block (DET: in canonical ray order, warps taking turns and each group of
// equal bins folded by its leader in lane order; otherwise warp-aggregated
// shared-memory atomics); then Eq. 3-6 noise per bin and I~ to HBM.
template <int DET>
__global__ void __launch_bounds__(512) k_bin(BinArgs a) {
    extern __shared__ float acc[];
    __shared__ SensorDev S;
    __shared__ SceneDev SC;
    __shared__ Unit U;
    __shared__ int s_unit, s_count;
    __shared__ float s_red[32];
    __shared__ float s_pat[kMaxCols];
    __shared__ int s_b0[kMaxCols + 1];   // per-beam fold: first local beam of each column
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const float alpha = __ldg(a.theta), gain = __ldg(a.theta + 1);
    for (int iter = 0;; ++iter) {
        int u;
        if (a.work_counter) {
            if (tid == 0) s_unit = atomicAdd(a.work_counter, 1);
            __syncthreads();
            u = s_unit;
        } else {
            if (iter > 0) break;
            u = blockIdx.x;
        }
        if (u >= a.n_units) break;
        if (tid == 0) load_unit(a, u, &S, &SC, &U);
        __syncthreads();
        const int cw = U.c1 - U.c0;
        const int i0 = first_beam_of_col(U.c0, S.nb, S.naz), i1 = first_beam_of_col(U.c1, S.nb, S.naz);
        const int64_t r0 = (int64_t)i0 * S.ne, r1 = (int64_t)i1 * S.ne;
        const int nbin = S.nr * cw;
        const sonar_hit* H = a.hits + S.hits_off;
        // Deterministic fold, per-beam form: warp w owns beams w, w + nw, ... of the
        // unit and folds each beam's rays in elevation order into that beam's own
        // row accumulator (one writer: no barriers); a bin then adds its column's
        // beams in beam order.  With one beam per column this is exactly the
        // sequential canonical-order fold.
        const int nbeam = i1 - i0;
        const bool per_beam = DET && S.fold_beams;
        float* accb = acc + nbin;
        int* list = reinterpret_cast<int*>(acc + nbin + (per_beam ? nbeam * S.nr : 0));
        if (per_beam) {
            for (int k = tid; k < nbeam * S.nr; k += nt) accb[k] = 0.0f;
            for (int c = tid; c <= cw; c += nt) s_b0[c] = first_beam_of_col(U.c0 + c, S.nb, S.naz) - i0;
        } else {
            for (int k = tid; k < nbin; k += nt) acc[k] = 0.0f;
        }
        __syncthreads();
        if (per_beam) {
            for (int bb = warp; bb < nbeam; bb += nw) {
                const sonar_hit* Hb = H + (int64_t)(i0 + bb) * S.ne;
                float* racc = accb + bb * S.nr;
                for (int jb = 0; jb < S.ne; jb += 32) {
                    const int j = jb + lane;
                    uint32_t row = kNoKey;
                    float score = 0.0f;
                    if (j < S.ne) {
                        const uint4 h = __ldg(reinterpret_cast<const uint4*>(Hb + j));
                        if (h.x != kNoKey) {
                            row = h.x / (uint32_t)S.naz;
                            int m = SC.mat_orig[h.y];
                            m = m < a.n_mat ? m : a.n_mat - 1;
                            score = __ldg(a.theta + 2 + m) * __uint_as_float(h.w) *
                                    expf(-2.0f * alpha * __uint_as_float(h.z)) * gain;
                        }
                    }
                    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, row);
                    if (row != kNoKey) {
                        const int leader = __ffs(peers) - 1;
                        float v = lane == leader ? racc[row] : 0.0f;
                        for (uint32_t m = peers; m; m &= m - 1) v += __shfl_sync(peers, score, __ffs(m) - 1);
                        if (lane == leader) racc[row] = v;
                    }
                }
            }
        }
        for (int64_t base = r0; base < (per_beam ? r0 : r1); base += nt) {
            const int64_t r = base + tid;
            uint32_t lkey = kNoKey;
            float score = 0.0f;
            if (r < r1) {
                const uint4 h = __ldg(reinterpret_cast<const uint4*>(H + r));
                if (h.x != kNoKey) {
                    const uint32_t br = h.x / (uint32_t)S.naz, ba = h.x - br * (uint32_t)S.naz;
                    lkey = br * (uint32_t)cw + (ba - (uint32_t)U.c0);
                    int m = SC.mat_orig[h.y];
                    m = m < a.n_mat ? m : a.n_mat - 1;
                    score = __ldg(a.theta + 2 + m) * __uint_as_float(h.w) *
                            expf(-2.0f * alpha * __uint_as_float(h.z)) * gain;
                }
            }
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, lkey);
            const int leader = __ffs(peers) - 1;
            if (DET) {
                for (int w = 0; w < nw; ++w) {
                    if (warp == w && lkey != kNoKey) {
                        float v = lane == leader ? acc[lkey] : 0.0f;
                        for (uint32_t m = peers; m; m &= m - 1) {
                            const float x = __shfl_sync(peers, score, __ffs(m) - 1);
                            v += x;
                        }
                        if (lane == leader) acc[lkey] = v;
                    }
                    __syncthreads();
                }
            } else {
                if (lkey != kNoKey) {
                    float v = 0.0f;
                    for (uint32_t m = peers; m; m &= m - 1) v += __shfl_sync(peers, score, __ffs(m) - 1);
                    if (lane == leader) atomicAdd(&acc[lkey], v);
                }
            }
        }
        __syncthreads();
        // Eq. 3-6 per bin.  Pass 1 visits every bin: Philox words, the additive
        // Rayleigh term, and the final value of bins without returns (P = 0 makes
        // the multiplicative term exactly 0); bins with returns are listed.  Pass 2
        // finishes the listed bins with the Gaussian multiplicative term.  (row,
        // col) advance incrementally: no division and no integer-to-float
        // conversion instruction in pass 1.
        const float dr = (S.rmax - S.rmin) / (float)S.nr, da = S.hfov / (float)S.naz;
        const float inv_rmax2 = 1.0f / (S.rmax * S.rmax);
        const float inv_sphi = 1.0f / a.params.sigma_phi;
        const float sig_sa = a.params.sigma_sa, sig_sm = a.params.sigma_sm;
        for (int c = tid; c < cw; c += nt) {
            const float pc = fmaf(small_u2f(U.c0 + c) + 0.5f, da, -0.5f * S.hfov);
            s_pat[c] = 0.5f * expf(-pc * pc * inv_sphi);
        }
        if (tid == 0) s_count = 0;
        __syncthreads();
        const int drow = nt / cw, dcol = nt - drow * cw;
        int row = tid / cw, col = tid - row * cw;
        const PhiloxKey K = philox_key(S.seed_lo, S.seed_hi);
        for (int k = tid; k < nbin; k += nt) {
            const uint32_t b = (uint32_t)(row * S.naz + U.c0 + col);
            float P;
            if (per_beam) {
                P = 0.0f;
                for (int bb = s_b0[col]; bb < s_b0[col + 1]; ++bb) P += accb[bb * S.nr + row];
            } else {
                P = acc[k];
            }
            const U4 x = bin_draws(b, S, K);
            const float w_sa = rayleigh_of(x, sig_sa);
            const float rc = fmaf(small_u2f(row) + 0.5f, dr, S.rmin);
            const float additive = rc * rc * inv_rmax2 * (1.0f + s_pat[col] * w_sa);
            if (a.binned) a.binned[S.polar_off + b] = P;
            if (P != 0.0f) {
                acc[k] = P;
                list[atomicAdd(&s_count, 1)] = k;
            } else {
                a.noised[S.polar_off + b] = additive;
                acc[k] = additive;
            }
            row += drow;
            col += dcol;
            if (col >= cw) { col -= cw; ++row; }
        }
        __syncthreads();
        const int nlist = s_count;
        for (int q = tid; q < nlist; q += nt) {
            const int k = list[q];
            const int rw = k / cw, cl = k - rw * cw;
            const uint32_t b = (uint32_t)(rw * S.naz + U.c0 + cl);
            const float P = acc[k];
            const U4 x = bin_draws(b, S, K);
            const float w_sa = rayleigh_of(x, sig_sa);
            const float rc = fmaf(small_u2f(rw) + 0.5f, dr, S.rmin);
            const float additive = rc * rc * inv_rmax2 * (1.0f + s_pat[cl] * w_sa);
            const float w_sm = gauss_of(x, sig_sm);
            const float In = P * (0.5f + w_sm) + additive;
            a.noised[S.polar_off + b] = In;
            acc[k] = In;
        }
        __syncthreads();
        if (a.params.normalise == 2) {
            // one maximum per unit for the whole-image normalisation; range-row
            // maxima are taken by the normalisation kernel from I~ itself
            float m = -CUDART_INF_F;
            for (int k = tid; k < nbin; k += nt) m = fmaxf(m, acc[k]);
            for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
            if (lane == 0) s_red[warp] = m;
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < nw; ++w) m = fmaxf(m, s_red[w]);
                atomicMax(a.rowmax + S.rowmax_off, ord_enc(fmaxf(m, s_red[0])));
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// phase 2a: range-wise normalisation, one warp per (sensor, range row)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float norm_value(float In, float m, int mode) {
    return (mode != 0 && m > 0.0f) ? In / m : In;
}

__global__ void __launch_bounds__(256) k_norm_rows(NormArgs a) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= a.total_rows) return;
    const SensorDev& s = a.sensors ? a.sensors[a.row_map[g]] : a.one;
    const int row = (int)(g - s.rowmax_off);
    const int naz = s.naz;
    const float* In = a.noised + s.polar_off + (int64_t)row * naz;
    float* out = a.polar + s.polar_off + (int64_t)row * naz;
    float m = 0.0f;
    if (((s.polar_off | naz) & 3) == 0 && naz <= 1024) {
        // 16-byte rows of up to 1024 bins: the row stays in registers between
        // the maximum and the division (one read of I~)
        const int n4 = naz >> 2;
        const float4* In4 = reinterpret_cast<const float4*>(In);
        float4* out4 = reinterpret_cast<float4*>(out);
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int q = lane + 32 * k;
            v[k] = q < n4 ? __ldg(In4 + q) : make_float4(-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F);
        }
        if (a.normalise == 1) {
            m = -CUDART_INF_F;
#pragma unroll
            for (int k = 0; k < 8; ++k) m = fmaxf(fmaxf(m, fmaxf(v[k].x, v[k].y)), fmaxf(v[k].z, v[k].w));
            for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        } else if (a.normalise == 2) {
            m = ord_dec(a.gmax[s.rowmax_off]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int q = lane + 32 * k;
            if (q < n4)
                out4[q] = make_float4(norm_value(v[k].x, m, a.normalise), norm_value(v[k].y, m, a.normalise),
                                      norm_value(v[k].z, m, a.normalise), norm_value(v[k].w, m, a.normalise));
        }
        return;
    }
    if (a.normalise == 1) {
        m = -CUDART_INF_F;
        for (int j = lane; j < naz; j += 32) m = fmaxf(m, In[j]);
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    } else if (a.normalise == 2) {
        m = ord_dec(a.gmax[s.rowmax_off]);
    }
    for (int j = lane; j < naz; j += 32) out[j] = norm_value(In[j], m, a.normalise);
}

// ---------------------------------------------------------------------------
// phase 2b: fan resample of the normalised image
// ---------------------------------------------------------------------------

// Where fan pixel `pix` samples the polar image: x = index of bin (ia, ja),
// y = (ib != ia ? naz : 0) << 1 | (jb != ja), z, w = the bilinear weights wr,
// wa (bit patterns); x = 0xFFFFFFFF outside the fan.  Bilinear over bin
// centres, clamped to the edge bins.
__device__ __forceinline__ uint4 fan_coord(const SensorDev& s, int64_t pix) {
    int v, u;
    if ((int64_t)s.fan_w * s.fan_h < (1ll << 31)) {
        v = (int)((uint32_t)pix / (uint32_t)s.fan_w);
        u = (int)pix - v * s.fan_w;
    } else {
        v = (int)(pix / s.fan_w);
        u = (int)(pix - (int64_t)v * s.fan_w);
    }
    const float inv_scale = 1.0f / s.fan_scale;
    const float x = ((float)u + 0.5f - 0.5f * (float)s.fan_w) * inv_scale;
    const float y = ((float)s.fan_h - (float)v - 0.5f) * inv_scale;
    const float r = sqrtf(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
    const float phi = atan2f(x, y);
    if (r < s.rmin || r > s.rmax || fabsf(phi) > 0.5f * s.hfov) return make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
    const float fr = __fsub_rn(__fmul_rn(r - s.rmin, s.inv_dr), 0.5f);
    const float fa = __fsub_rn(__fmul_rn(phi + 0.5f * s.hfov, (float)s.naz / s.hfov), 0.5f);
    const float i0f = floorf(fr), j0f = floorf(fa);
    const float wr = fr - i0f, wa = fa - j0f;
    const int i0 = (int)i0f, j0 = (int)j0f;
    const int ia = min(max(i0, 0), s.nr - 1), ib = min(max(i0 + 1, 0), s.nr - 1);
    const int ja = min(max(j0, 0), s.naz - 1), jb = min(max(j0 + 1, 0), s.naz - 1);
    return make_uint4((uint32_t)(ia * s.naz + ja), ((ib != ia ? (uint32_t)s.naz : 0u) << 1) | (jb != ja ? 1u : 0u),
                      __float_as_uint(wr), __float_as_uint(wa));
}

// The fan value at coordinates c over polar image P (explicit roundings: the
// table and the direct path give the same bits).
__device__ __forceinline__ float fan_blend(uint4 c, const float* P) {
    if (c.x == 0xFFFFFFFFu) return 0.0f;
    const uint32_t dj = c.y & 1u, dn = c.y >> 1;
    const float* q = P + c.x;
    const float wr = __uint_as_float(c.z), wa = __uint_as_float(c.w);
    const float ua = 1.0f - wa, ur = 1.0f - wr;
    const float top = __fadd_rn(__fmul_rn(ua, q[0]), __fmul_rn(wa, q[dj]));
    const float bot = __fadd_rn(__fmul_rn(ua, q[dn]), __fmul_rn(wa, q[dn + dj]));
    return __fadd_rn(__fmul_rn(ur, top), __fmul_rn(wr, bot));
}

// One block = a kFanSide x kFanSide square of one sensor's fan (a square maps
// to a compact patch of the polar image, so its gathers stay in cache); lane
// x of a 64-thread row takes column x, rows step by 4.  A sensor with a
// coordinate table reads its pixels' coordinates from it.
__global__ void __launch_bounds__(256) k_fan_tiles(FanArgs a) {
    __shared__ SensorDev S;
    __shared__ int s_sq;
    if (threadIdx.x == 0) {
        if (a.block_map) {
            const int2 m = a.block_map[blockIdx.x];
            S = a.sensors[m.x];
            s_sq = m.y;
        } else {
            S = a.one;
            s_sq = blockIdx.x;
        }
    }
    __syncthreads();
    const int sx = (S.fan_w + kFanSide - 1) / kFanSide;
    const int u = (s_sq % sx) * kFanSide + (threadIdx.x & (kFanSide - 1));
    const int v0 = (s_sq / sx) * kFanSide + (threadIdx.x / kFanSide);
    if (u >= S.fan_w) return;
    const float* P = a.polar + S.polar_off;
    float* F = a.fan + S.fan_off;
    const uint4* lut = S.fan_lut;
#pragma unroll 4
    for (int k = 0; k < kFanSide; k += 256 / kFanSide) {
        const int v = v0 + k;
        if (v >= S.fan_h) break;
        const int64_t pix = (int64_t)v * S.fan_w + u;
        F[pix] = fan_blend(lut ? __ldg(lut + pix) : fan_coord(S, pix), P);
    }
}

// The fan of the frames that share one coordinate table, in the same squares:
// one thread reads a pixel's table entry once and resamples that pixel for up
// to kFanGroup frames (a frame whose geometry no longer matches the table
// computes its own coordinates).
__global__ void __launch_bounds__(256) k_fan_group(FanGroupArgs a) {
    __shared__ SensorDev M[kFanGroup];
    __shared__ int4 s_m;
    __shared__ int s_w, s_h;
    __shared__ const uint4* s_lut;
    if (threadIdx.x == 0) {
        s_m = a.block_map[blockIdx.x];
        const SensorDev& o = a.sensors[s_m.x];
        s_w = o.fan_w;
        s_h = o.fan_h;
        s_lut = o.fan_lut;
    }
    __syncthreads();
    const int nm = s_m.w - s_m.z;
    constexpr int kWords = (int)(sizeof(SensorDev) / 4);
    for (int i = threadIdx.x; i < nm * kWords; i += blockDim.x) {
        const int q = i / kWords;
        reinterpret_cast<uint32_t*>(M)[i] =
            reinterpret_cast<const uint32_t*>(a.sensors + a.members[s_m.z + q])[i - q * kWords];
    }
    __syncthreads();
    const int w = s_w, h = s_h;
    const int sx = (w + kFanSide - 1) / kFanSide;
    const int u = (s_m.y % sx) * kFanSide + (threadIdx.x & (kFanSide - 1));
    const int v0 = (s_m.y / sx) * kFanSide + (threadIdx.x / kFanSide);
    if (u >= w) return;
    const uint4* lut = s_lut;
#pragma unroll 1
    for (int k = 0; k < kFanSide; k += 256 / kFanSide) {
        const int v = v0 + k;
        if (v >= h) break;
        const int64_t pix = (int64_t)v * w + u;
        const uint4 c = lut ? __ldg(lut + pix) : fan_coord(M[0], pix);
#pragma unroll
        for (int q = 0; q < kFanGroup; ++q) {
            if (q < nm) {
                const uint4 cq = M[q].fan_lut ? c : fan_coord(M[q], pix);
                a.fan[M[q].fan_off + pix] = fan_blend(cq, a.polar + M[q].polar_off);
            }
        }
    }
}

// Fills the coordinate table of each owner sensor (one block = kFanTile pixels).
__global__ void __launch_bounds__(256) k_fan_lut(FanLutArgs a) {
    __shared__ SensorDev S;
    __shared__ int64_t s_base;
    __shared__ uint4* s_lut;
    if (threadIdx.x == 0) {
        const int2 m = a.block_map[blockIdx.x];
        S = a.sensors[m.x];
        s_base = (int64_t)m.y * kFanTile;
        s_lut = a.luts[m.x];
    }
    __syncthreads();
    const int64_t n = (int64_t)S.fan_w * S.fan_h;
#pragma unroll 1
    for (int k = 0; k < kFanTile / 256; ++k) {
        const int64_t pix = s_base + k * 256 + threadIdx.x;
        if (pix < n) s_lut[pix] = fan_coord(S, pix);
    }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------

// Group terms of the normalisation Jacobian: m, argmax (lowest index on
// ties) and c = sum G I~ / m^2.  Mode 1: one warp per range row; mode 2: one
// block per sensor image.
__global__ void k_adj_rows(const SensorDev* sensors, const int32_t* row_map, SensorDev one, int n_sensors,
                           int64_t total, int mode, const float* noised, const float* grad, RowInfo* info) {
    const int lane = threadIdx.x & 31;
    __shared__ float s_m[32];
    __shared__ int s_a[32];
    __shared__ ff s_d[32];
    if (mode == 1) {
        const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (g >= total) return;
        const SensorDev& s = sensors ? sensors[row_map[g]] : one;
        const int row = (int)(g - s.rowmax_off);
        const float* In = noised + s.polar_off + (int64_t)row * s.naz;
        const float* G = grad + s.polar_off + (int64_t)row * s.naz;
        float m = -CUDART_INF_F;
        int am = 0x7FFFFFFF;
        float dl = 0.0f;                      // per-lane partial of sum G I~ (few terms)
        if (((s.polar_off | s.naz) & 3) == 0) {
            // 16-byte rows: each lane takes 4 consecutive bins per load, in index order
            const float4* In4 = reinterpret_cast<const float4*>(In);
            const float4* G4 = reinterpret_cast<const float4*>(G);
#pragma unroll 4
            for (int q = lane; q < (s.naz >> 2); q += 32) {
                const float4 x = __ldg(In4 + q), y = __ldg(G4 + q);
                const int j = q << 2;
                if (x.x > m) { m = x.x; am = j; }
                if (x.y > m) { m = x.y; am = j + 1; }
                if (x.z > m) { m = x.z; am = j + 2; }
                if (x.w > m) { m = x.w; am = j + 3; }
                dl = fmaf(y.x, x.x, dl);
                dl = fmaf(y.y, x.y, dl);
                dl = fmaf(y.z, x.z, dl);
                dl = fmaf(y.w, x.w, dl);
            }
        } else {
            for (int j = lane; j < s.naz; j += 32) {
                const float x = In[j];
                if (x > m) { m = x; am = j; }
                dl = fmaf(G[j], x, dl);
            }
        }
        // lane partials added across the warp in float-float (error-free
        // two-sums on the FP32 pipes: FP64 would cost more than the row's loads)
        ff dot{dl, 0.0f};
        for (int o = 16; o; o >>= 1) {
            const float m2 = __shfl_xor_sync(0xFFFFFFFFu, m, o);
            const int a2 = __shfl_xor_sync(0xFFFFFFFFu, am, o);
            if (m2 > m || (m2 == m && a2 < am)) { m = m2; am = a2; }
            const ff d2{__shfl_xor_sync(0xFFFFFFFFu, dot.hi, o), __shfl_xor_sync(0xFFFFFFFFu, dot.lo, o)};
            dot = ff_add(dot, d2);
        }
        if (lane == 0) {
            RowInfo r;
            r.m = m;
            r.valid = m > 0.0f;
            r.c = r.valid ? (__fadd_rn(dot.hi, dot.lo) / m) / m : 0.0f;
            r.arg = row * s.naz + am;
            info[g] = r;
        }
    } else {
        const int si = blockIdx.x;
        if (si >= total) return;
        const SensorDev& s = sensors ? sensors[si] : one;
        const int64_t n = (int64_t)s.nr * s.naz;
        const float* In = noised + s.polar_off;
        const float* G = grad + s.polar_off;
        float m = -CUDART_INF_F;
        int am = 0x7FFFFFFF;
        ff dot{0.0f, 0.0f};   // float-float: products exact (FMA), sums error-free
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const float x = In[j], y = G[j];
            if (x > m) { m = x; am = (int)j; }
            const float p = __fmul_rn(y, x);
            dot = ff_add(dot, ff{p, fmaf(y, x, -p)});
        }
        for (int o = 16; o; o >>= 1) {
            const float m2 = __shfl_xor_sync(0xFFFFFFFFu, m, o);
            const int a2 = __shfl_xor_sync(0xFFFFFFFFu, am, o);
            if (m2 > m || (m2 == m && a2 < am)) { m = m2; am = a2; }
            const ff d2{__shfl_xor_sync(0xFFFFFFFFu, dot.hi, o), __shfl_xor_sync(0xFFFFFFFFu, dot.lo, o)};
            dot = ff_add(dot, d2);
        }
        const int w = threadIdx.x >> 5;
        if (lane == 0) { s_m[w] = m; s_a[w] = am; s_d[w] = dot; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                if (s_m[k] > m || (s_m[k] == m && s_a[k] < am)) { m = s_m[k]; am = s_a[k]; }
                dot = ff_add(dot, s_d[k]);
            }
            RowInfo r;
            r.m = m;
            r.valid = m > 0.0f;
            r.c = r.valid ? (__fadd_rn(dot.hi, dot.lo) / m) / m : 0.0f;
            r.arg = am;
            info[s.rowmax_off] = r;
        }
    }
}

// Per-ray gather of dL/dP and accumulation of dtheta over a unit of rays,
// reading the hit records (stored by the forward, or recomputed by the ray-cast
// kernel just before: bitwise the same records).
// Deterministic: each unit's sums go to its own row of `partials` (material
// sums per warp in lane order, warp slabs added in warp order, alpha/gain per
// thread then in a fixed tree); k_adj_final adds the rows in a fixed order.
// A unit holds a few hundred rays: its sums are FP32 (float-float across
// lanes), its row of partials FP64.
__global__ void __launch_bounds__(512) k_adjoint(AdjArgs a) {
    extern __shared__ double slab_d[];   // [n_warps][n_mat] (FP32 sums; sized in doubles by the host)
    float* slab = reinterpret_cast<float*>(slab_d);
    __shared__ SensorDev S;
    __shared__ SceneDev SC;
    __shared__ AdjUnit U;
    __shared__ int s_unit;
    __shared__ ff s_ag[2][32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int nm = a.n_mat, nq = nm + 2;
    const float alpha = __ldg(a.theta), gain = __ldg(a.theta + 1);
    const int mode = a.params.normalise;
    for (int iter = 0;; ++iter) {
        int u;
        if (a.work_counter) {
            if (tid == 0) s_unit = atomicAdd(a.work_counter, 1);
            __syncthreads();
            u = s_unit;
        } else {
            if (iter > 0) break;
            u = blockIdx.x;
        }
        if (u >= a.n_units) break;
        if (tid == 0) {
            if (a.units) {
                U = a.units[u];
                S = a.sensors[U.sensor];
                SC = a.scenes[S.scene];
            } else {
                S = a.one;
                SC = a.one_scene;
                U.sensor = 0;
                U.r0 = u * a.chunk;
                U.r1 = min(U.r0 + a.chunk, a.one.nb * a.one.ne);
            }
        }
        for (int k = tid; k < nw * nm; k += nt) slab[k] = 0.0f;
        __syncthreads();
        const PhiloxKey K = philox_key(S.seed_lo, S.seed_hi);
        float acc_a = 0.0f, acc_g = 0.0f;
        for (int base = U.r0; base < U.r1; base += nt) {
            const int r = base + tid;
            bool valid = false;
            int mat = 0;
            float v_mu = 0.0f;
            if (r < U.r1) {
                const uint4 h = __ldg(reinterpret_cast<const uint4*>(a.hits + S.hits_off + r));
                const uint32_t key = h.x, orig = h.y;
                const float rr = __uint_as_float(h.z), cf = __uint_as_float(h.w);
                if (key != kNoKey) {
                    if (key >= (uint32_t)(S.nr * S.naz) || orig >= (uint32_t)SC.n_tris) {
                        atomicOr(a.err, SONAR_DEVERR_INDEX);
                    } else {
                        const float G = a.grad[S.polar_off + key];
                        float gI = G;
                        if (mode != 0) {
                            const RowInfo ri = a.rowinfo[S.rowmax_off + (mode == 1 ? (int)(key / S.naz) : 0)];
                            if (ri.valid) gI = G / ri.m - ((int)key == ri.arg ? ri.c : 0.0f);
                        }
                        const float gP = gI * (0.5f + w_sm_of(key, S, a.params.sigma_sm, K));
                        mat = SC.mat_orig[orig];
                        mat = mat < nm ? mat : nm - 1;
                        const float mu = __ldg(a.theta + 2 + mat);
                        const float ca = gP * cf * expf(-2.0f * alpha * rr);
                        v_mu = ca * gain;
                        acc_a = fmaf(ca * gain * mu, -2.0f * rr, acc_a);
                        acc_g = fmaf(ca, mu, acc_g);
                        valid = true;
                    }
                }
            }
            // material sums of this warp: one leader per material, lanes in order
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, valid ? mat : -1);
            if (valid) {
                float sum = 0.0f;
                for (uint32_t m = peers; m; m &= m - 1) sum += __shfl_sync(peers, v_mu, __ffs(m) - 1);
                if (lane == __ffs(peers) - 1) slab[warp * nm + mat] += sum;
            }
        }
        ff da{acc_a, 0.0f}, dg{acc_g, 0.0f};
        for (int o = 16; o; o >>= 1) {
            da = ff_add(da, ff{__shfl_down_sync(0xFFFFFFFFu, da.hi, o), __shfl_down_sync(0xFFFFFFFFu, da.lo, o)});
            dg = ff_add(dg, ff{__shfl_down_sync(0xFFFFFFFFu, dg.hi, o), __shfl_down_sync(0xFFFFFFFFu, dg.lo, o)});
        }
        if (lane == 0) { s_ag[0][warp] = da; s_ag[1][warp] = dg; }
        __syncthreads();
        double* out = a.partials + (int64_t)u * nq;
        for (int m = tid; m < nm; m += nt) {
            ff v{0.0f, 0.0f};
            for (int w = 0; w < nw; ++w) v = ff_add(v, ff{slab[w * nm + m], 0.0f});
            out[2 + m] = (double)v.hi + (double)v.lo;
        }
        if (tid == 0) {
            ff va{0.0f, 0.0f}, vg{0.0f, 0.0f};
            for (int w = 0; w < nw; ++w) { va = ff_add(va, s_ag[0][w]); vg = ff_add(vg, s_ag[1][w]); }
            out[0] = (double)va.hi + (double)va.lo;
            out[1] = (double)vg.hi + (double)vg.lo;
        }
        __syncthreads();
    }
}

// dtheta[q] = sum over units of partials[u][q]: a fixed strided split over the
// threads, then a fixed tree.
__global__ void __launch_bounds__(256) k_adj_final(const double* partials, int n_units, int nq, float* dtheta) {
    __shared__ double red[256];
    const int q = blockIdx.x;
    double v = 0.0;
    for (int u = threadIdx.x; u < n_units; u += 256) v += partials[(int64_t)u * nq + q];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) dtheta[q] = (float)red[0];
}

// ---------------------------------------------------------------------------
// counters
// ---------------------------------------------------------------------------

__global__ void k_popcount(const uint32_t* bits, int64_t words, unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x)
        c += __popc(bits[w]);
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
// DVL (Sec. III-A-3): four-beam Janus ranges, least-squares velocity, rate
// ---------------------------------------------------------------------------

// Closest hit along one ray (any origin and direction) by a per-thread walk
// of the 4-wide hierarchy: certified FP32 Moller-Trumbore, undecided tests
// decided exactly in float-float on the FP32 direction; ties go to the lower
// caller index.  Returns the distance (+inf for a miss).
__device__ float closest_distance(const SceneDev& sc, float3 o, float3 d, float tmax, uint32_t* err) {
    if (sc.root == kEmpty) return CUDART_INF_F;
    const float tiny = 1e-20f;
    const float3 inv = f3(1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                          1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                          1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    const float3 oinv = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    const float of[3] = {o.x, o.y, o.z};
    const ff dff[3] = {ff{d.x, 0.0f}, ff{d.y, 0.0f}, ff{d.z, 0.0f}};
    int32_t stack[kStackMax];
    int sp = 0;
    float best_t = tmax;
    uint32_t best_id = 0xFFFFFFFFu;
    int32_t node = sc.root;
    while (node != kEmpty) {
        if (node < 0) {
            const int32_t x = ~node;
            const int32_t first = x >> 3, count = (x & 7) + 1;
            for (int k = 0; k < count; ++k) {
                const int32_t f = first + k;
                if (f >= sc.n_tris) {
                    atomicOr(err, SONAR_DEVERR_INDEX);
                    break;
                }
                const float4* tp = sc.tris + 3 * (int64_t)f;
                const float4 va = __ldg(tp), vb = __ldg(tp + 1), vc = __ldg(tp + 2);
                float t;
                const int r = mt32(o, d, va, vb, vc, t);
                if (r == 0) continue;
                if (r == 2) {
                    ff D, T;
                    if (!mt_ff(of, dff, va, vb, vc, D, T)) continue;
                    t = T.hi / D.hi;
                }
                const uint32_t id = __float_as_uint(vb.w);
                if (t < best_t || (t == best_t && id < best_id)) {
                    best_t = t;
                    best_id = id;
                }
            }
            node = sp > 0 ? stack[--sp] : kEmpty;
            continue;
        }
        const float4* pn = sc.nodes + 8 * (int64_t)node;
        const float4 lx = __ldg(pn), hx = __ldg(pn + 1), ly = __ldg(pn + 2), hy = __ldg(pn + 3);
        const float4 lz = __ldg(pn + 4), hz = __ldg(pn + 5);
        const int4 ch = __ldg(reinterpret_cast<const int4*>(pn + 6));
        const float tcut = best_t * 1.00002f;
        const float lxs[4] = {lx.x, lx.y, lx.z, lx.w}, hxs[4] = {hx.x, hx.y, hx.z, hx.w};
        const float lys[4] = {ly.x, ly.y, ly.z, ly.w}, hys[4] = {hy.x, hy.y, hy.z, hy.w};
        const float lzs[4] = {lz.x, lz.y, lz.z, lz.w}, hzs[4] = {hz.x, hz.y, hz.z, hz.w};
        const int32_t hs[4] = {ch.x, ch.y, ch.z, ch.w};
        uint32_t key[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float t0 = fmaf(lxs[c], inv.x, -oinv.x), t1 = fmaf(hxs[c], inv.x, -oinv.x);
            float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
            t0 = fmaf(lys[c], inv.y, -oinv.y); t1 = fmaf(hys[c], inv.y, -oinv.y);
            lo = fmaxf(lo, fminf(t0, t1)); hi = fminf(hi, fmaxf(t0, t1));
            t0 = fmaf(lzs[c], inv.z, -oinv.z); t1 = fmaf(hzs[c], inv.z, -oinv.z);
            lo = fmaxf(fmaxf(lo, fminf(t0, t1)), 0.0f); hi = fminf(fminf(hi, fmaxf(t0, t1)), tcut);
            const bool hit = hs[c] != kEmpty && lo <= hi * 1.0000005f;
            key[c] = hit ? ((__float_as_uint(lo) & ~3u) | (uint32_t)c) : 0xFFFFFFFFu;
        }
#define SONAR_USORT(x, y)                                \
        {                                                \
            const uint32_t mn = min(key[x], key[y]);     \
            key[y] = max(key[x], key[y]);                \
            key[x] = mn;                                 \
        }
        SONAR_USORT(0, 1) SONAR_USORT(2, 3) SONAR_USORT(0, 2) SONAR_USORT(1, 3) SONAR_USORT(1, 2)
#undef SONAR_USORT
        const int nhit = (key[0] != 0xFFFFFFFFu) + (key[1] != 0xFFFFFFFFu) + (key[2] != 0xFFFFFFFFu) +
                         (key[3] != 0xFFFFFFFFu);
        if (nhit == 0) {
            node = sp > 0 ? stack[--sp] : kEmpty;
            continue;
        }
        if (sp + nhit - 1 > kStackMax) {   // cannot happen for a checked depth: give up the ray
            atomicOr(err, SONAR_DEVERR_STACK);
            return CUDART_INF_F;
        }
        for (int c = nhit - 1; c >= 1; --c) {
            const uint32_t k = key[c] & 3u;
            stack[sp++] = k == 0 ? hs[0] : k == 1 ? hs[1] : k == 2 ? hs[2] : hs[3];
        }
        const uint32_t k = key[0] & 3u;
        node = k == 0 ? hs[0] : k == 1 ? hs[1] : k == 2 ? hs[2] : hs[3];
    }
    return best_id == 0xFFFFFFFFu ? CUDART_INF_F : best_t;
}

// A standard normal from two Philox words: the cosine branch of Box-Muller.
__device__ __forceinline__ float normal_of(uint32_t a, uint32_t b) {
    const float u2 = fmaf((float)b, 0x1p-32f, 0x1p-32f);
    return sqrt_nonneg(neg2log_u(a)) * cospif(2.0f * u2);
}

// Four lanes per pose, lane k casting beam k; the group's first lane fits the
// velocity by least squares over the valid beams (Cramer's rule on the 3 x 3
// normal equations) and writes the pose's outputs.
__global__ void __launch_bounds__(128) k_dvl(DvlArgs a) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = g >> 2;
    const int k = (int)(g & 3);
    const int lane = threadIdx.x & 31, base = lane & ~3;
    const unsigned grp = 0xFu << base;
    const bool live = p < a.n;
    float range = CUDART_INF_F, u = 0.0f;
    bool valid = false;
    if (live) {
        const float* q = a.pose + 12 * p;
        const float3 o = f3(q[0], q[1], q[2]);
        const float* R = q + 3;
        const float bx = a.beam[k][0], by = a.beam[k][1], bz = a.beam[k][2];
        float3 d = f3(fmaf(R[0], bx, fmaf(R[1], by, R[2] * bz)), fmaf(R[3], bx, fmaf(R[4], by, R[5] * bz)),
                      fmaf(R[6], bx, fmaf(R[7], by, R[8] * bz)));
        range = closest_distance(a.scene, o, d, CUDART_INF_F, a.err);
        valid = range >= a.r_min && range <= a.r_max;
        // sensor-frame velocity R^T v and this beam's radial velocity with noise
        const float* vw = a.vel_world + 3 * p;
        const float vs0 = fmaf(R[0], vw[0], fmaf(R[3], vw[1], R[6] * vw[2]));
        const float vs1 = fmaf(R[1], vw[0], fmaf(R[4], vw[1], R[7] * vw[2]));
        const float vs2 = fmaf(R[2], vw[0], fmaf(R[5], vw[1], R[8] * vw[2]));
        const U4 x = philox10(U4{(uint32_t)p, (uint32_t)((uint64_t)p >> 32), 2u, (uint32_t)(k >> 1)},
                              a.seed_lo, a.seed_hi);
        const float w = (k & 1) ? normal_of(x.z, x.w) : normal_of(x.x, x.y);
        u = fmaf(bx, vs0, fmaf(by, vs1, bz * vs2)) + a.sigma_b * w;
        a.ranges[4 * p + k] = range;
    }
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    float rr[4], uu[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        rr[j] = __shfl_sync(0xFFFFFFFFu, range, base + j);
        uu[j] = __shfl_sync(0xFFFFFFFFu, u, base + j);
    }
    if (!live || k != 0) return;
    const unsigned bits = (vm & grp) >> base;
    const int nvalid = __popc(bits);
    float A[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, y[3] = {0.f, 0.f, 0.f};
    float far = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!((bits >> j) & 1u)) continue;
        far = fmaxf(far, rr[j]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            y[r] = fmaf(a.beam[j][r], uu[j], y[r]);
#pragma unroll
            for (int c = 0; c < 3; ++c) A[r][c] = fmaf(a.beam[j][r], a.beam[j][c], A[r][c]);
        }
    }
    int32_t flags = (int32_t)bits;
    float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
    const float det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                      A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                      A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (nvalid >= a.min_beams && det != 0.0f) {
        const float id = 1.0f / det;
        v0 = (y[0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (y[1] * A[2][2] - A[1][2] * y[2]) +
              A[0][2] * (y[1] * A[2][1] - A[1][1] * y[2])) * id;
        v1 = (A[0][0] * (y[1] * A[2][2] - A[1][2] * y[2]) - y[0] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
              A[0][2] * (A[1][0] * y[2] - y[1] * A[2][0])) * id;
        v2 = (A[0][0] * (A[1][1] * y[2] - y[1] * A[2][1]) - A[0][1] * (A[1][0] * y[2] - y[1] * A[2][0]) +
              y[0] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) * id;
        flags |= 16;
    }
    a.vel[3 * p] = v0;
    a.vel[3 * p + 1] = v1;
    a.vel[3 * p + 2] = v2;
    a.flags[p] = flags;
    a.period[p] = (flags & 16) ? fmaf(a.t1, far, a.t0) : a.t_lost;
}

// Emission schedule: one thread per vehicle walks its steps (a measurement at
// step 0, then max(1, ceil(period / dt)) steps after each measurement).
__global__ void k_dvl_schedule(const float* period, int64_t n_veh, int64_t n_steps, float dt, int32_t* emit) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_veh) return;
    const float* P = period + v * n_steps;
    int32_t* E = emit + v * n_steps;
    for (int64_t s = 0; s < n_steps; ++s) E[s] = 0;
    int64_t s = 0;
    while (s < n_steps) {
        E[s] = 1;
        const float q = ceilf(P[s] / dt);
        s += q >= 1.0f ? (int64_t)q : 1;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

void set_kernel_attributes() {
    cudaFuncSetAttribute(k_bin<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    cudaFuncSetAttribute(k_bin<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

cudaError_t launch_trig(const SensorDev* sensors, const SensorDev& one, int n_sensors, int max_angles,
                        cudaStream_t st) {
    const dim3 grid((unsigned)((max_angles + 127) / 128), (unsigned)n_sensors);
    k_trig<<<grid, 128, 0, st>>>(sensors, one);
    return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs& a, int blocks, int occupancy, cudaStream_t st) {
    if (blocks > 0) {
        if (occupancy >= 8) k_trace<32, false><<<blocks, 32, 0, st>>>(a);
        else k_trace<4, false><<<blocks, 32, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_bin(const BinArgs& a, int det, int grid, int block, size_t smem, cudaStream_t st) {
    if (det) k_bin<1><<<grid, block, smem, st>>>(a);
    else k_bin<0><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

int bin_blocks_per_sm(int det, int block, size_t smem) {
    int n = 0;
    const void* f = det ? (const void*)k_bin<1> : (const void*)k_bin<0>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_norm(const NormArgs& a, cudaStream_t st) {
    const int64_t threads = a.total_rows * 32;
    k_norm_rows<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fan_tiles(const FanArgs& a, int blocks, cudaStream_t st) {
    if (blocks > 0) k_fan_tiles<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fan_group(const FanGroupArgs& a, int blocks, cudaStream_t st) {
    if (blocks > 0) k_fan_group<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fan_lut(const FanLutArgs& a, int blocks, cudaStream_t st) {
    if (blocks > 0) k_fan_lut<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_rows(const SensorDev* sensors, const int32_t* row_map, const SensorDev& one, int n_sensors,
                            int64_t total_groups, int normalise, const float* noised,
                            const float* grad, RowInfo* info, cudaStream_t st) {
    if (normalise == 1) {
        const int64_t threads = total_groups * 32;
        k_adj_rows<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(sensors, row_map, one, n_sensors,
                                                                      total_groups, 1, noised, grad, info);
    } else if (normalise == 2) {
        k_adj_rows<<<(unsigned)total_groups, 1024, 0, st>>>(sensors, row_map, one, n_sensors, total_groups, 2,
                                                            noised, grad, info);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjArgs& a, int grid, int block, size_t smem, float* dtheta, cudaStream_t st) {
    k_adjoint<<<grid, block, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_final<<<a.n_mat + 2, 256, 0, st>>>(a.partials, a.n_units, a.n_mat + 2, dtheta);
    return cudaGetLastError();
}

int adjoint_blocks_per_sm(int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)k_adjoint, block, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_dvl(const DvlArgs& a, cudaStream_t st) {
    if (a.n > 0) k_dvl<<<(unsigned)((4 * a.n + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dvl_schedule(const float* period, int64_t n_veh, int64_t n_steps, float dt, int32_t* emit,
                                cudaStream_t st) {
    if (n_veh > 0 && n_steps > 0) k_dvl_schedule<<<(unsigned)((n_veh + 127) / 128), 128, 0, st>>>(period, n_veh, n_steps, dt, emit);
    return cudaGetLastError();
}

cudaError_t launch_stats(const SensorDev& s, const SceneDev& sc, const sonar_params& p,
                         const TraceCounters& tc, uint32_t* err, cudaStream_t st) {
    TraceArgs a{};
    a.one = s;
    a.one_scene = sc;
    a.n_sensors = 1;
    a.params = p;
    a.err = err;
    a.tc = tc;
    if (s.trace_blocks > 0) k_trace<4, true><<<s.trace_blocks, 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_popcount(const uint32_t* bits, int64_t words, unsigned long long* out, cudaStream_t st) {
    k_popcount<<<1024, 256, 0, st>>>(bits, words, out);
    return cudaGetLastError();
}

}  // namespace sonar
