// Sonar ray casting (OceanSim, arXiv 2503.01074, Sec. III-A-2).
//
// k_trig              float-float sin/cos tables of each sensor's beam azimuths
//                     and elevations (FP64 once per sensor).
// k_trace             one ray per thread, warps on compact beam x elevation
//                     patches: ray generation -> closest hit (LBVH walk,
//                     Moller-Trumbore) -> range/azimuth bin -> 16-byte hit record.
//                     The STATS variant counts node visits and triangle tests and
//                     marks the nodes and triangles it touches.
// k_popcount          counts the marked nodes and triangles.
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
#include "devmath.cuh"

namespace sonar {
namespace {

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


// Two consecutive float4 of a node (32 bytes, 32-byte aligned: nodes are
// 128-byte lines) in one 256-bit read-only load, so that a node visit takes
// four load instructions instead of seven.
__device__ __forceinline__ void ld_node_pair(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
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
    // a batch block whose entries were built for the sensor's current fields of
    // view has nothing to do (block-uniform; only later launches read the table)
    if (s.trig_stamp && s.trig_stamp[blockIdx.x] == s.trig_version) return;
    if (s.trig_stamp && threadIdx.x == 0) s.trig_stamp[blockIdx.x] = s.trig_version;
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


// ---------------------------------------------------------------------------
// trace: one ray per thread, hit record out
// ---------------------------------------------------------------------------

// A float twice, as the packed pair operand of fma.rn.f32x2.
__device__ __forceinline__ unsigned long long pk2(float v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
    return r;
}
// (d0, d1) = (a0, a1) * b + c element by element in one packed FP32 FMA
// (sm_100 and later), each element rounded exactly like fmaf
__device__ __forceinline__ void fma2(float a0, float a1, unsigned long long b, unsigned long long c, float& d0,
                                     float& d1) {
    asm("{\n\t.reg .b64 ra, rd;\n\tmov.b64 ra, {%2, %3};\n\tfma.rn.f32x2 rd, ra, %4, %5;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1) : "f"(a0), "f"(a1), "l"(b), "l"(c));
}
// Sorts W child keys ascending in registers: a 5-comparator network for 4,
// Batcher's odd-even merge sort (19 comparators) for 8.
template <int W>
__device__ __forceinline__ void sort_keys(uint32_t (&key)[W]) {
#define SONAR_USORT(x, y)                            \
    {                                                \
        const uint32_t mn = min(key[x], key[y]);     \
        key[y] = max(key[x], key[y]);                \
        key[x] = mn;                                 \
    }
    if constexpr (W == 4) {
        SONAR_USORT(0, 1) SONAR_USORT(2, 3) SONAR_USORT(0, 2) SONAR_USORT(1, 3) SONAR_USORT(1, 2)
    } else {
        SONAR_USORT(0, 1) SONAR_USORT(2, 3) SONAR_USORT(4, 5) SONAR_USORT(6, 7)
        SONAR_USORT(0, 2) SONAR_USORT(1, 3) SONAR_USORT(4, 6) SONAR_USORT(5, 7)
        SONAR_USORT(1, 2) SONAR_USORT(5, 6)
        SONAR_USORT(0, 4) SONAR_USORT(1, 5) SONAR_USORT(2, 6) SONAR_USORT(3, 7)
        SONAR_USORT(2, 4) SONAR_USORT(3, 5)
        SONAR_USORT(1, 2) SONAR_USORT(3, 4) SONAR_USORT(5, 6)
    }
#undef SONAR_USORT
}

// The handle in slot k (0 <= k < W) of a node's handles held in registers.
template <int W>
__device__ __forceinline__ int32_t child_at(const int32_t (&hs)[W], uint32_t k) {
    if constexpr (W == 4) {
        return k == 0 ? hs[0] : k == 1 ? hs[1] : k == 2 ? hs[2] : hs[3];
    } else {
        const int32_t h01 = (k & 1) ? hs[1] : hs[0], h23 = (k & 1) ? hs[3] : hs[2];
        const int32_t h45 = (k & 1) ? hs[5] : hs[4], h67 = (k & 1) ? hs[7] : hs[6];
        const int32_t h03 = (k & 2) ? h23 : h01, h47 = (k & 2) ? h67 : h45;
        return (k & 4) ? h47 : h03;
    }
}

// Each block is one warp on a tile of tb beams x (32 / tb) elevations of one
// sensor: lane l traces beam i0 + l % tb, elevation j0 + l / tb, so that the
// warp's rays sample a compact patch of the field of view.  (One-warp blocks
// free their slot as soon as their rays are done.)  Records go to their
// canonical index i * n_elev + j.
//
// The walk over the W-wide hierarchy (W = 4, or 8 for launches too small to
// fill the GPU, where fewer dependent node loads per ray matter more than the
// extra box tests per visit) is a while-while loop: a lane descends
// nearest child first, pushing the other entered children; a lane that
// reaches a leaf parks it and keeps descending until every active lane of the
// warp holds one, so that the triangle tests run together.  A lane whose ray
// is finished writes its record at once and idles until the warp is done.
// With STATS the kernel also counts node visits and triangle tests and marks
// the nodes and triangles it touches (records are then not written).
template <int MINB, bool STATS, int W>
__global__ void __launch_bounds__(32, MINB) k_trace(TraceArgs a) {
    __shared__ SensorDev S;
    __shared__ SceneDev SC;
    if (a.zero_word && blockIdx.x == 0 && threadIdx.x == 0) *a.zero_word = 0;   // read by the next launch only
    int tile;
    if (a.sensors) {
        // the warp copies the sensor and scene descriptors word by word, both at
        // once (the map carries the scene index): one round trip after the map
        const int4 m = a.block_map[blockIdx.x];
        const uint32_t* s_src = reinterpret_cast<const uint32_t*>(a.sensors + m.x);
        const uint32_t* c_src = reinterpret_cast<const uint32_t*>(a.scenes + m.z);
        constexpr int kSW = (int)(sizeof(SensorDev) / 4), kCW = (int)(sizeof(SceneDev) / 4);
        for (int i = threadIdx.x; i < kSW; i += 32) reinterpret_cast<uint32_t*>(&S)[i] = __ldg(s_src + i);
        for (int i = threadIdx.x; i < kCW; i += 32) reinterpret_cast<uint32_t*>(&SC)[i] = __ldg(c_src + i);
        tile = m.y;
    } else {
        if (threadIdx.x == 0) {
            S = a.one;
            SC = a.one_scene;
        }
        tile = blockIdx.x;
    }
    __syncthreads();
    const int tb = S.tb, te = 32 / S.tb;
    const int tiles_b = (S.nb + tb - 1) / tb;
    const int ty = tile / tiles_b, tx = tile - ty * tiles_b;
    const int lane = threadIdx.x;
    const int ri = tx * tb + (lane % tb);
    const int rj = ty * te + lane / tb;
    const SceneDev& sc = SC;
    const sonar_params& p = a.params;
    // without clipping any finite distance counts: 3e38 stands for infinity so
    // that the box cut below (1.00002 times the best distance) stays finite
    const float tlimit = p.clip_tmax ? S.rmax : 3.0e38f;
    const float3 o = f3(S.pos[0], S.pos[1], S.pos[2]);
    const bool inside = ri < S.nb && rj < S.ne;
    const float3 d = inside ? ray_dir32(S, ri, rj) : f3(0.0f, 0.0f, 1.0f);
    const float tiny = 1e-20f;
    const float3 inv = f3(1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                          1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                          1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    const float3 oinv = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    // (inv, inv) and (-o inv, -o inv) per axis as packed pairs for the box tests
    const unsigned long long ivx = pk2(inv.x), ivy = pk2(inv.y), ivz = pk2(inv.z);
    const unsigned long long novx = pk2(-oinv.x), novy = pk2(-oinv.y), novz = pk2(-oinv.z);
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
                const float4* pn = W == 4 ? sc.nodes + 8 * (int64_t)node : sc.nodes8 + 16 * (int64_t)node;
                if (STATS) {
                    ++visits;
                    atomicOr(a.tc.node_bits + (node >> 5), 1u << (node & 31));
                }
                const float tcut = best_t * 1.00002f;
                // sort key per child: entry distance bits (>= 0, so integer order
                // is distance order) with the child slot in the low bits; a
                // missed child sorts last as 0xFFFFFFFF
                uint32_t key[W];
                int32_t hs[W];
#pragma unroll
                for (int half = 0; half < W / 4; ++half) {   // a 4-wide node, or the halves of an 8-wide one
                    float4 lx, hx, ly, hy, lz, hz, chf, unused;
                    ld_node_pair(pn + 8 * half, lx, hx);
                    ld_node_pair(pn + 8 * half + 2, ly, hy);
                    ld_node_pair(pn + 8 * half + 4, lz, hz);
                    ld_node_pair(pn + 8 * half + 6, chf, unused);
                    hs[4 * half + 0] = __float_as_int(chf.x);
                    hs[4 * half + 1] = __float_as_int(chf.y);
                    hs[4 * half + 2] = __float_as_int(chf.z);
                    hs[4 * half + 3] = __float_as_int(chf.w);
                    // per axis, the (lo, hi) planes of children 0, 1 | 2, 3
                    const float lxs[4] = {lx.x, lx.z, hx.x, hx.z}, hxs[4] = {lx.y, lx.w, hx.y, hx.w};
                    const float lys[4] = {ly.x, ly.z, hy.x, hy.z}, hys[4] = {ly.y, ly.w, hy.y, hy.w};
                    const float lzs[4] = {lz.x, lz.z, hz.x, hz.z}, hzs[4] = {lz.y, lz.w, hz.y, hz.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float t0, t1;
                        fma2(lxs[c], hxs[c], ivx, novx, t0, t1);
                        float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
                        fma2(lys[c], hys[c], ivy, novy, t0, t1);
                        lo = fmaxf(lo, fminf(t0, t1)); hi = fminf(hi, fmaxf(t0, t1));
                        fma2(lzs[c], hzs[c], ivz, novz, t0, t1);
                        lo = fmaxf(fmaxf(lo, fminf(t0, t1)), 0.0f); hi = fminf(fminf(hi, fmaxf(t0, t1)), tcut);
                        // an empty slot's box lies at +inf on every axis: along an axis
                        // the ray travels in the + direction its entry distance is +inf,
                        // and if it travels in the - direction along all three its exit
                        // distance is -inf; the exit is also at most tcut, which is
                        // finite, so an empty slot never passes and needs no handle check
                        const bool hit = lo <= hi * 1.0000005f;
                        key[4 * half + c] =
                            hit ? ((__float_as_uint(lo) & ~(uint32_t)(W - 1)) | (uint32_t)(4 * half + c)) : 0xFFFFFFFFu;
                    }
                }
                sort_keys<W>(key);
                int nhit = 0;
#pragma unroll
                for (int c = 0; c < W; ++c) nhit += key[c] != 0xFFFFFFFFu;
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
                    for (int c = W - 1; c >= 1; --c) {
                        if (c < nhit) stack[sp++] = child_at<W>(hs, key[c] & (uint32_t)(W - 1));
                    }
                    node = child_at<W>(hs, key[0] & (uint32_t)(W - 1));
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
// counters
// ---------------------------------------------------------------------------

__global__ void k_popcount(const uint32_t* bits, int64_t words, unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x)
        c += __popc(bits[w]);
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_trig(const SensorDev* sensors, const SensorDev& one, int n_sensors, int max_angles,
                        cudaStream_t st) {
    const dim3 grid((unsigned)((max_angles + 127) / 128), (unsigned)n_sensors);
    k_trig<<<grid, 128, 0, st>>>(sensors, one);
    return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs& a, int blocks, int occupancy, cudaStream_t st) {
    if (blocks > 0) {
        const bool cap = occupancy & kTraceCap;
        // one sensor's launch on a scene without an 8-wide tree walks the 4-wide
        // one (a batch's variant is checked against all its scenes on the host)
        const bool wide = (occupancy & kTraceWide) && (a.sensors || a.one_scene.nodes8);
        if (wide) {
            if (cap) k_trace<32, false, 8><<<blocks, 32, 0, st>>>(a);
            else k_trace<4, false, 8><<<blocks, 32, 0, st>>>(a);
        } else {
            if (cap) k_trace<32, false, 4><<<blocks, 32, 0, st>>>(a);
            else k_trace<4, false, 4><<<blocks, 32, 0, st>>>(a);
        }
    }
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
    if (s.trace_blocks > 0) {
        if ((s.occ & kTraceWide) && sc.nodes8) k_trace<4, true, 8><<<s.trace_blocks, 32, 0, st>>>(a);
        else k_trace<4, true, 4><<<s.trace_blocks, 32, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_popcount(const uint32_t* bits, int64_t words, unsigned long long* out, cudaStream_t st) {
    k_popcount<<<1024, 256, 0, st>>>(bits, words, out);
    return cudaGetLastError();
}

}  // namespace sonar
