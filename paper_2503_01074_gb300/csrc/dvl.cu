// DVL kernels (OceanSim, arXiv 2503.01074, Sec. III-A-3): four-beam Janus ranges by
// a per-thread walk of the 4-wide hierarchy, least-squares velocity, range-
// dependent ping period and dropout, and the per-vehicle emission schedule.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "sonar_host.h"
#include "sonar_internal.cuh"
#include "devmath.cuh"

namespace sonar {
namespace {

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
        // per axis, the (lo, hi) planes of children 0, 1 | 2, 3
        const float lxs[4] = {lx.x, lx.z, hx.x, hx.z}, hxs[4] = {lx.y, lx.w, hx.y, hx.w};
        const float lys[4] = {ly.x, ly.z, hy.x, hy.z}, hys[4] = {ly.y, ly.w, hy.y, hy.w};
        const float lzs[4] = {lz.x, lz.z, hz.x, hz.z}, hzs[4] = {lz.y, lz.w, hz.y, hz.w};
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

cudaError_t launch_dvl(const DvlArgs& a, cudaStream_t st) {
    if (a.n > 0) k_dvl<<<(unsigned)((4 * a.n + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dvl_schedule(const float* period, int64_t n_veh, int64_t n_steps, float dt, int32_t* emit,
                                cudaStream_t st) {
    if (n_veh > 0 && n_steps > 0) k_dvl_schedule<<<(unsigned)((n_veh + 127) / 128), 128, 0, st>>>(period, n_veh, n_steps, dt, emit);
    return cudaGetLastError();
}

}  // namespace sonar
