// LBVH construction for the sonar geometry query (OceanSim Sec. III-A-2:
// the scene is queried by ray casting; this builds the acceleration structure).
//
//   1. validate + centroid bounds     one thread per triangle, block-reduced atomics
//   2. Morton codes                   63-bit keys (21 bits per axis) of triangle centroids
//   3. radix sort                     stable LSD, 8-bit digits, histogram / scan / scatter
//   4. Karras hierarchy               one thread per internal node (Karras, HPG 2012)
//   5. bottom-up refit                leaf-to-root climb, second visitor merges boxes
//   6. packing                        runs of <= kLeafMax triangles collapsed into
//                                     leaves; 48-byte triangles
//   7. wide collapse                  twice, into a 4-wide and an 8-wide tree: a
//                                     bottom-up dynamic programme gives each subtree's
//                                     least SAH cost in 1..W child slots; top-down,
//                                     one level per pass, each node takes the children
//                                     it chose; SoA nodes (128 or 256 bytes) in
//                                     breadth-first order
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sonar_internal.cuh"
#include "sonar_host.h"

namespace sonar {
namespace {

constexpr int kThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kThreads * kRsItems;   // keys per sort block

// ---------------------------------------------------------------------------
// 1. validation and centroid bounds
// ---------------------------------------------------------------------------

struct BuildStats {
    uint32_t flags;        // 1: index out of range, 2: negative material, 4: non-finite vertex
    int32_t max_mat;
    uint32_t lo[3], hi[3]; // ordered-encoded centroid bounds
};

__device__ __forceinline__ float3 load_v(const float* v, int32_t i) {
    return make_float3(v[3 * (int64_t)i], v[3 * (int64_t)i + 1], v[3 * (int64_t)i + 2]);
}

__global__ void k_validate(const float* verts, int64_t nv, const int32_t* tris, const int32_t* mat,
                           int64_t nt, BuildStats* st) {
    __shared__ uint32_t s_lo[3], s_hi[3], s_flags;
    __shared__ int32_t s_mat;
    if (threadIdx.x < 3) { s_lo[threadIdx.x] = 0xFFFFFFFFu; s_hi[threadIdx.x] = 0u; }
    if (threadIdx.x == 0) { s_flags = 0; s_mat = -1; }
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) {
        const int32_t a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        uint32_t f = 0;
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) f |= 1u;
        const int32_t m = mat[t];
        if (m < 0) f |= 2u;
        if (!f) {
            const float3 p = load_v(verts, a), q = load_v(verts, b), r = load_v(verts, c);
            const bool fin = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(q.x) &&
                             isfinite(q.y) && isfinite(q.z) && isfinite(r.x) && isfinite(r.y) &&
                             isfinite(r.z);
            if (!fin) {
                f |= 4u;
            } else {
                const float cx = (p.x + q.x + r.x) * (1.0f / 3.0f);
                const float cy = (p.y + q.y + r.y) * (1.0f / 3.0f);
                const float cz = (p.z + q.z + r.z) * (1.0f / 3.0f);
                atomicMin(&s_lo[0], ord_enc(cx)); atomicMax(&s_hi[0], ord_enc(cx));
                atomicMin(&s_lo[1], ord_enc(cy)); atomicMax(&s_hi[1], ord_enc(cy));
                atomicMin(&s_lo[2], ord_enc(cz)); atomicMax(&s_hi[2], ord_enc(cz));
            }
        }
        if (f) atomicOr(&s_flags, f);
        atomicMax(&s_mat, m);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&st->lo[threadIdx.x], s_lo[threadIdx.x]);
        atomicMax(&st->hi[threadIdx.x], s_hi[threadIdx.x]);
    }
    if (threadIdx.x == 0) {
        if (s_flags) atomicOr(&st->flags, s_flags);
        atomicMax(&st->max_mat, s_mat);
    }
}

// ---------------------------------------------------------------------------
// 2. Morton codes
// ---------------------------------------------------------------------------

__global__ void k_morton(const float* verts, const int32_t* tris, int64_t nt, const BuildStats* st,
                         uint64_t* keys, uint32_t* vals) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const float3 p = load_v(verts, tris[3 * t]), q = load_v(verts, tris[3 * t + 1]),
                 r = load_v(verts, tris[3 * t + 2]);
    const float c[3] = {(p.x + q.x + r.x) * (1.0f / 3.0f), (p.y + q.y + r.y) * (1.0f / 3.0f),
                        (p.z + q.z + r.z) * (1.0f / 3.0f)};
    // one scale for all axes (the largest extent): a flat scene (a seabed is
    // ~100 m wide and a few m high) then splits across its width first and in
    // height only at fine levels; per-axis scaling split it in height as early
    // as in x and y, into wide overlapping boxes (+30 % node visits per ray)
    uint32_t g[3];
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) ext = fmaxf(ext, ord_dec(st->hi[a]) - ord_dec(st->lo[a]));
    for (int a = 0; a < 3; ++a) {
        const float lo = ord_dec(st->lo[a]);
        float u = ext > 0.0f ? (c[a] - lo) / ext : 0.0f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        g[a] = (uint32_t)fminf(u * 2097152.0f, 2097151.0f);    // 21 bits
    }
    uint64_t key = 0;
    for (int b = 20; b >= 0; --b) {
        key = (key << 3) | ((uint64_t)((g[0] >> b) & 1u) << 2) | ((uint64_t)((g[1] >> b) & 1u) << 1) |
              (uint64_t)((g[2] >> b) & 1u);
    }
    keys[t] = key;
    vals[t] = (uint32_t)t;
}

// ---------------------------------------------------------------------------
// 3. stable LSD radix sort (8-bit digits)
// ---------------------------------------------------------------------------

__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, uint32_t* hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int k = 0; k < kRsItems; ++k) {
        const int64_t i = base + k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of a u32 array in three passes (chunk sums, scan of sums, apply).
constexpr int kScanChunk = kThreads * 16;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_sums(const uint32_t* in, int64_t n, uint32_t* sums) {
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * 16;
    uint32_t v = 0;
    for (int k = 0; k < 16; ++k)
        if (base + k < n) v += in[base + k];
    uint32_t total;
    block_exclusive_scan(v, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_top(uint32_t* sums, int64_t n) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < n ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, s_warp, total);
        const uint32_t carry = s_carry;
        if (i < n) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + total;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const uint32_t* in, int64_t n, const uint32_t* sums, uint32_t* out) {
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * 16;
    uint32_t loc[16];
    uint32_t v = 0;
    for (int k = 0; k < 16; ++k) {
        loc[k] = base + k < n ? in[base + k] : 0u;
        v += loc[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(v, s_warp, total) + sums[blockIdx.x];
    for (int k = 0; k < 16; ++k) {
        if (base + k < n) out[base + k] = run;
        run += loc[k];
    }
}

// Stable scatter: rounds of 256 consecutive keys; within a round, rank =
// (keys of the same digit in earlier warps) + (earlier lanes of this warp);
// rounds advance a running per-digit offset.
__global__ void k_rs_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                             int64_t n, int shift, const uint32_t* offs, int nblocks) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[kThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    for (int w = 0; w < kThreads / 32; ++w) wc[w][threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int k = 0; k < kRsItems; ++k) {
        const int64_t i = base + k * kThreads + threadIdx.x;
        const bool ok = i < n;
        const uint64_t key = ok ? kin[i] : 0ull;
        const uint32_t val = ok ? vin[i] : 0u;
        const uint32_t digit = ok ? (uint32_t)((key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, digit);
        const uint32_t rank = __popc(peers & lt);
        if (ok && rank == 0) wc[warp][digit] = __popc(peers);
        __syncthreads();
        {
            uint32_t r = run[threadIdx.x];
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t c = wc[w][threadIdx.x];
                wc[w][threadIdx.x] = r;
                r += c;
            }
            run[threadIdx.x] = r;
        }
        __syncthreads();
        if (ok) {
            const uint32_t pos = wc[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        for (int w = 0; w < kThreads / 32; ++w) wc[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 4. Karras hierarchy
// ---------------------------------------------------------------------------

// Length of the common prefix of keys i and j; equal keys are told apart by
// their indices (64 + common prefix of i and j); -1 outside [0, n).
__device__ __forceinline__ int delta(const uint64_t* k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t a = k[i], b = k[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

// child[2p], child[2p+1]: internal c >= 0 or leaf ~c; parent[p] for internal
// nodes, parent[n - 1 + i] for leaf i; range[p] = covered leaves [lo, hi].
__global__ void k_karras(const uint64_t* keys, int64_t n, int32_t* child, int32_t* parent,
                         int2* range) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = delta(keys, n, i, i + 1) > delta(keys, n, i, i - 1) ? 1 : -1;
    const int dmin = delta(keys, n, i, i - d);
    int64_t lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(keys, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    const int32_t left = lo == gamma ? ~(int32_t)gamma : (int32_t)gamma;
    const int32_t right = hi == gamma + 1 ? ~(int32_t)(gamma + 1) : (int32_t)(gamma + 1);
    child[2 * i] = left;
    child[2 * i + 1] = right;
    parent[left >= 0 ? left : (n - 1) + ~left] = (int32_t)i;
    parent[right >= 0 ? right : (n - 1) + ~right] = (int32_t)i;
    range[i] = make_int2((int)lo, (int)hi);
    if (i == 0) parent[0] = -1;
}

// ---------------------------------------------------------------------------
// 5. bottom-up refit
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tri_box(const float* verts, const int32_t* tris, uint32_t orig,
                                        float3& lo, float3& hi) {
    const float3 p = load_v(verts, tris[3 * (int64_t)orig]), q = load_v(verts, tris[3 * (int64_t)orig + 1]),
                 r = load_v(verts, tris[3 * (int64_t)orig + 2]);
    lo = make_float3(fminf(p.x, fminf(q.x, r.x)), fminf(p.y, fminf(q.y, r.y)), fminf(p.z, fminf(q.z, r.z)));
    hi = make_float3(fmaxf(p.x, fmaxf(q.x, r.x)), fmaxf(p.y, fmaxf(q.y, r.y)), fmaxf(p.z, fmaxf(q.z, r.z)));
}

__device__ __forceinline__ void child_box(int32_t c, const float* verts, const int32_t* tris,
                                          const uint32_t* vals, const float4* blo, const float4* bhi,
                                          float3& lo, float3& hi, int& h) {
    if (c < 0) {
        tri_box(verts, tris, vals[~c], lo, hi);
        h = 0;
    } else {
        const float4 a = __ldcg(blo + c), b = __ldcg(bhi + c);
        lo = make_float3(a.x, a.y, a.z);
        hi = make_float3(b.x, b.y, b.z);
        h = __float_as_int(b.w);
    }
}

__global__ void k_refit(const float* verts, const int32_t* tris, const uint32_t* vals, int64_t n,
                        const int32_t* child, const int32_t* parent, int32_t* visits, float4* blo,
                        float4* bhi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = parent[(n - 1) + i];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&visits[p], 1) == 0) return;   // the other child is still on its way
        float3 l0, h0, l1, h1;
        int e0, e1;
        child_box(child[2 * p], verts, tris, vals, blo, bhi, l0, h0, e0);
        child_box(child[2 * p + 1], verts, tris, vals, blo, bhi, l1, h1, e1);
        const int h = 1 + (e0 > e1 ? e0 : e1);
        __stcg(blo + p, make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.0f));
        __stcg(bhi + p, make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), __int_as_float(h)));
        __threadfence();
        p = parent[p];
    }
}

// ---------------------------------------------------------------------------
// 6. packing
// ---------------------------------------------------------------------------

__global__ void k_pack_nodes(const float* verts, const int32_t* tris, const uint32_t* vals, int64_t n,
                             const int32_t* child, const int2* range, const float4* blo,
                             const float4* bhi, float pad, float4* nodes) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n - 1) return;
    for (int side = 0; side < 2; ++side) {
        const int32_t c = child[2 * p + side];
        float3 lo, hi;
        int32_t handle;
        if (c < 0) {
            tri_box(verts, tris, vals[~c], lo, hi);
            handle = leaf_handle(~c, 1);
        } else {
            const float4 a = blo[c], b = bhi[c];
            lo = make_float3(a.x, a.y, a.z);
            hi = make_float3(b.x, b.y, b.z);
            const int2 r = range[c];
            const int cnt = r.y - r.x + 1;
            handle = cnt <= kLeafMax ? leaf_handle(r.x, cnt) : c;
        }
        nodes[4 * p + 2 * side] = make_float4(lo.x - pad, lo.y - pad, lo.z - pad, __int_as_float(handle));
        nodes[4 * p + 2 * side + 1] = make_float4(hi.x + pad, hi.y + pad, hi.z + pad, 0.0f);
    }
}

__global__ void k_pack_tris(const float* verts, const int32_t* tris, const int32_t* mat,
                            const uint32_t* vals, int64_t n, float4* out, int32_t* mat_orig) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t o = vals[k];
    const float3 p = load_v(verts, tris[3 * (int64_t)o]), q = load_v(verts, tris[3 * (int64_t)o + 1]),
                 r = load_v(verts, tris[3 * (int64_t)o + 2]);
    const int32_t m = mat[o];
    out[3 * k] = make_float4(p.x, p.y, p.z, __int_as_float(m));
    out[3 * k + 1] = make_float4(q.x, q.y, q.z, __uint_as_float(o));
    out[3 * k + 2] = make_float4(r.x, r.y, r.z, 0.0f);
    mat_orig[o] = m;
}

// ---- 4-wide collapse (top-down, one level of the 4-wide tree per pass) ----
// A child under construction is a side of a binary node: x = 2 * p + side, its
// box and handle at pairs[2 x] (lo, handle bits) and pairs[2 x + 1] (hi).

__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

constexpr float kSahTri = 0.7f;   // SAH cost of a triangle test relative to a wide-node visit
// ---- SAH-driven collapse: a bottom-up dynamic programme over the binary tree ----
// cost(x, k): the least SAH cost of the subtree at side x (a leaf run or a
// binary node) when it may take up to k (1..W) child slots of the W-wide node
// above it.  One slot: the side itself, a leaf (area x triangles x kSahTri) or
// a W-wide node (area + the cost of its subtree spread over W slots); k slots:
// the better of that and opening the node, its two sides sharing the k slots.
// dec[p] keeps, for k = 2..W, the split of p's slots between its sides
// (SplitBits<W> bits each, from bit 0) and whether p is better opened (one bit
// each above the splits).  cost holds W floats per binary node.
template <int W>
struct Wide {
    static constexpr int kSplitBits = W == 8 ? 3 : 2;
    static constexpr int kOpenBit = kSplitBits * (W - 1);
    __host__ __device__ static constexpr int split(int32_t d, int k) {
        return (d >> (kSplitBits * (k - 2))) & ((1 << kSplitBits) - 1);
    }
    __host__ __device__ static constexpr bool opened(int32_t d, int k) { return (d >> (kOpenBit + k - 2)) & 1; }
};

template <int W>
__device__ __forceinline__ float side_cost(const float4* pairs, const float* cost, int64_t x, int k) {
    const float4 lo = pairs[2 * x], hi = pairs[2 * x + 1];
    const int32_t h = __float_as_int(lo.w);
    if (h < 0) return half_area(lo, hi) * kSahTri * (float)(((~h) & 7) + 1);
    return __ldcg(cost + (int64_t)W * h + (k - 1));
}

template <int W>
__global__ void k_sah_dp(int64_t n, const int32_t* parent, int32_t* visits, const float4* pairs, float* cost,
                         int32_t* dec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = parent[(n - 1) + i];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&visits[p], 1) == 0) return;   // the other child is still on its way
        float S0[W + 1], S1[W + 1];
        for (int k = 1; k <= W; ++k) {
            S0[k] = side_cost<W>(pairs, cost, 2 * (int64_t)p, k);
            S1[k] = side_cost<W>(pairs, cost, 2 * (int64_t)p + 1, k);
        }
        // opening p into m slots: the best split j | m - j
        float open[W + 1];
        int split[W + 1];
        for (int m = 2; m <= W; ++m) {
            open[m] = 3.0e38f;
            split[m] = 1;
            for (int j = 1; j < m; ++j) {
                const float v = S0[j] + S1[m - j];
                if (v < open[m]) { open[m] = v; split[m] = j; }
            }
        }
        const float4 l0 = pairs[4 * (int64_t)p], h0 = pairs[4 * (int64_t)p + 1];
        const float4 l1 = pairs[4 * (int64_t)p + 2], h1 = pairs[4 * (int64_t)p + 3];
        const float4 ul = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.0f);
        const float4 uh = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.0f);
        // one slot: p as a W-wide node of its own, its two sides sharing the W slots
        const float wide = half_area(ul, uh) + open[W];
        __stcg(cost + (int64_t)W * p, wide);
        int32_t d = 0;
        for (int k = 2; k <= W; ++k) {
            const bool opened = open[k] < wide;
            __stcg(cost + (int64_t)W * p + (k - 1), opened ? open[k] : wide);
            d |= (split[k] << (Wide<W>::kSplitBits * (k - 2))) | (opened ? (1 << (Wide<W>::kOpenBit + k - 2)) : 0);
        }
        dec[p] = d;
        __threadfence();
        p = parent[p];
    }
}

// The children of entry e (internal binary node q[e]) from the programme: p's
// W slots split between its sides, each side taking its slots as a leaf, a
// W-wide node (one slot) or opened further.  Every side keeps at least one
// slot, so at most W sides are pending at once.
template <int W>
__global__ void k_collapse_pick(const int32_t* q, int64_t nq, const float4* pairs, const int32_t* dec,
                                int32_t* picks, uint32_t* nint) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nq) return;
    const int32_t p = q[e];
    int32_t c[W];
    for (int k = 0; k < W; ++k) c[k] = -1;
    int cnt = 0;
    // work list of (side, slots)
    int32_t ws[W + 1];
    int wk[W + 1];
    int nw = 0;
    {
        const int j = Wide<W>::split(dec[p], W);
        ws[nw] = 2 * p + 1; wk[nw++] = W - j;
        ws[nw] = 2 * p;     wk[nw++] = j;
    }
    while (nw > 0) {
        const int32_t x = ws[--nw];
        const int k = wk[nw];
        const int32_t h = __float_as_int(pairs[2 * (int64_t)x].w);
        if (h < 0 || k < 2 || !Wide<W>::opened(dec[h], k)) {
            c[cnt++] = x;
            continue;
        }
        const int j = Wide<W>::split(dec[h], k);
        ws[nw] = 2 * h + 1; wk[nw++] = k - j;
        ws[nw] = 2 * h;     wk[nw++] = j;
    }
    uint32_t ni = 0;
    for (int k = 0; k < W; ++k) {
        picks[W * e + k] = c[k];
        if (c[k] >= 0 && __float_as_int(pairs[2 * (int64_t)c[k]].w) >= 0) ++ni;
    }
    nint[e] = ni;
}

// The next level's entries: the internal children, in entry and slot order.
template <int W>
__global__ void k_collapse_enqueue(const int32_t* picks, const uint32_t* prefix, int64_t nq, const float4* pairs,
                                   int32_t* q_next) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nq) return;
    uint32_t r = prefix[e];
    for (int k = 0; k < W; ++k) {
        const int32_t x = picks[W * e + k];
        if (x < 0) continue;
        const int32_t h = __float_as_int(pairs[2 * (int64_t)x].w);
        if (h >= 0) q_next[r++] = h;
    }
}

// Writes the W-wide nodes of one level: entry e is node base + e, W / 4
// halves in the 4-wide layout; its r-th internal child is node base_next +
// prefix[e] + r.  Empty slots hold an inverted box that no ray enters and the
// empty handle.
template <int W>
__global__ void k_collapse_write(const int32_t* picks, const uint32_t* prefix, int64_t nq, int64_t base,
                                 int64_t base_next, const float4* pairs, float4* nodes) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nq) return;
    uint32_t r = prefix[e];
    for (int half = 0; half < W / 4; ++half) {
        float lo[3][4], hi[3][4];
        int32_t hh[4];
        for (int k = 0; k < 4; ++k) {
            const int32_t x = picks[W * e + 4 * half + k];
            if (x < 0) {
                for (int a = 0; a < 3; ++a) lo[a][k] = hi[a][k] = __int_as_float(0x7F800000);
                hh[k] = kEmpty;
                continue;
            }
            const float4 l = pairs[2 * (int64_t)x], h = pairs[2 * (int64_t)x + 1];
            lo[0][k] = l.x; lo[1][k] = l.y; lo[2][k] = l.z;
            hi[0][k] = h.x; hi[1][k] = h.y; hi[2][k] = h.z;
            const int32_t c = __float_as_int(l.w);
            hh[k] = c >= 0 ? (int32_t)(base_next + r++) : c;
        }
        float4* o = nodes + 2 * W * (base + e) + 8 * half;
        for (int a = 0; a < 3; ++a) {   // per axis: (lo, hi) of children 0, 1 | 2, 3
            o[2 * a] = make_float4(lo[a][0], hi[a][0], lo[a][1], hi[a][1]);
            o[2 * a + 1] = make_float4(lo[a][2], hi[a][2], lo[a][3], hi[a][3]);
        }
        o[6] = make_float4(__int_as_float(hh[0]), __int_as_float(hh[1]), __int_as_float(hh[2]),
                           __int_as_float(hh[3]));
        o[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Temporary device buffers of one build, freed in stream order on exit.
struct BuildScratch {
    static constexpr int kMax = 32;
    cudaStream_t st;
    void* ptrs[kMax] = {};
    int n = 0;
    cudaError_t err = cudaSuccess;
    template <class T>
    T* get(size_t count) {
        void* p = nullptr;
        if (n >= kMax) err = cudaErrorMemoryAllocation;   // more buffers than slots: refuse, never overflow
        if (err == cudaSuccess) err = cudaMallocAsync(&p, count * sizeof(T) + 16, st);
        if (err != cudaSuccess) return nullptr;
        ptrs[n++] = p;
        return (T*)p;
    }
    ~BuildScratch() {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], st);
    }
};

// Buffers of the wide collapse, sized for the widest tree and shared by both.
struct CollapseScratch {
    float* cost;       // [8 n] SAH cost per binary node and slot count
    int32_t* dec;      // [n] the programme's decisions per binary node
    int32_t *qa, *qb;  // [n] binary nodes of the current / next level
    int32_t* picks;    // [8 n] per wide node: the binary sides in its slots
    uint32_t *nint, *prefix, *fsums;
};

// One W-wide tree from the binary hierarchy in `pairs`: the cost programme
// bottom-up, then top-down one level per pass (picks and prefixes of every
// level kept, indexed by wide node), the nodes written once their count is
// known.  *nodes_out is a new allocation owned by the caller.
template <int W>
cudaError_t collapse_tree(const CollapseScratch& C, int64_t n, const int32_t* parent, int32_t* visits,
                          const float4* pairs, cudaStream_t st, float4** nodes_out, int64_t* count_out,
                          int* depth_out) {
    *nodes_out = nullptr;
    cudaError_t e = cudaMemsetAsync(visits, 0, sizeof(int32_t) * (n - 1), st);
    if (e != cudaSuccess) return e;
    k_sah_dp<W><<<blocks_for(n, kThreads), kThreads, 0, st>>>(n, parent, visits, pairs, C.cost, C.dec);
    const int32_t zero = 0;
    e = cudaMemcpyAsync(C.qa, &zero, sizeof zero, cudaMemcpyHostToDevice, st);
    std::vector<int64_t> lbase, lcount;
    int64_t base = 0, nq = 1;
    int32_t *qa = C.qa, *qb = C.qb;
    while (e == cudaSuccess && nq > 0) {
        if (base + nq > n) { e = cudaErrorInvalidValue; break; }   // cannot happen: nodes are distinct
        lbase.push_back(base);
        lcount.push_back(nq);
        const int64_t ch = (nq + kScanChunk - 1) / kScanChunk;
        k_collapse_pick<W><<<blocks_for(nq, kThreads), kThreads, 0, st>>>(qa, nq, pairs, C.dec, C.picks + W * base,
                                                                          C.nint + base);
        k_scan_sums<<<(unsigned)ch, kThreads, 0, st>>>(C.nint + base, nq, C.fsums);
        k_scan_top<<<1, 1024, 0, st>>>(C.fsums, ch);
        k_scan_apply<<<(unsigned)ch, kThreads, 0, st>>>(C.nint + base, nq, C.fsums, C.prefix + base);
        k_collapse_enqueue<W><<<blocks_for(nq, kThreads), kThreads, 0, st>>>(C.picks + W * base, C.prefix + base,
                                                                             nq, pairs, qb);
        uint32_t last[2] = {0, 0};
        e = cudaMemcpyAsync(&last[0], C.prefix + base + nq - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&last[1], C.nint + base + nq - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        base += nq;
        nq = (int64_t)last[0] + last[1];
        int32_t* t = qa; qa = qb; qb = t;
    }
    if (e != cudaSuccess) return e;
    const int64_t count = base;
    float4* nodes = nullptr;
    e = cudaMalloc(&nodes, sizeof(float4) * 2 * W * std::max<int64_t>(count, 1));
    if (e != cudaSuccess) return e;
    for (size_t L = 0; L < lbase.size(); ++L) {
        const int64_t nxt = L + 1 < lbase.size() ? lbase[L + 1] : count;
        k_collapse_write<W><<<blocks_for(lcount[L], kThreads), kThreads, 0, st>>>(
            C.picks + W * lbase[L], C.prefix + lbase[L], lcount[L], lbase[L], nxt, pairs, nodes);
    }
    *nodes_out = nodes;
    *count_out = count;
    *depth_out = (int)lbase.size();
    return cudaGetLastError();
}

sonar_status build_scene(const float* verts, int64_t nv, const int32_t* tris, const int32_t* mat,
                         int64_t nt, cudaStream_t st, SceneStore* out, std::string* msg) {
    *out = SceneStore{};
    out->n_tris = nt;
    out->max_mat = -1;
    if (nt == 0) {
        out->root = kEmpty;
        return SONAR_OK;
    }
    BuildScratch S{st};
    BuildStats* d_stats = S.get<BuildStats>(1);
    if (!d_stats) { *msg = "out of device memory (build statistics)"; return SONAR_ERR_OOM; }
    BuildStats init{};
    init.flags = 0;
    init.max_mat = -1;
    for (int a = 0; a < 3; ++a) { init.lo[a] = 0xFFFFFFFFu; init.hi[a] = 0u; }
    if (cudaMemcpyAsync(d_stats, &init, sizeof init, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        *msg = "cudaMemcpyAsync failed"; return SONAR_ERR_CUDA;
    }
    k_validate<<<blocks_for(nt, kThreads), kThreads, 0, st>>>(verts, nv, tris, mat, nt, d_stats);
    BuildStats hs{};
    cudaError_t e = cudaMemcpyAsync(&hs, d_stats, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { *msg = std::string("validation failed: ") + cudaGetErrorString(e); return SONAR_ERR_CUDA; }
    if (hs.flags & 1u) { *msg = "triangle vertex index out of range"; return SONAR_ERR_ARG; }
    if (hs.flags & 2u) { *msg = "negative material id"; return SONAR_ERR_ARG; }
    if (hs.flags & 4u) { *msg = "non-finite vertex coordinate"; return SONAR_ERR_ARG; }
    out->max_mat = hs.max_mat;

    // box padding: covers the difference between the FP32 traversal ray and
    // the exact ray, so that the FP32 box test never culls an exact hit
    float ext = 0.0f, mag = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const uint32_t lo = hs.lo[a], hi = hs.hi[a];
        auto dec = [](uint32_t v) {
            uint32_t b = (v & 0x80000000u) ? (v & 0x7FFFFFFFu) : ~v;
            float f;
            memcpy(&f, &b, 4);
            return f;
        };
        const float l = dec(lo), h = dec(hi);
        ext = fmaxf(ext, h - l);
        mag = fmaxf(mag, fmaxf(fabsf(l), fabsf(h)));
    }
    const float pad = fmaxf(1e-5f * (ext + mag), 1e-6f);

    const int64_t n = nt;
    uint64_t* k0 = S.get<uint64_t>(n);
    uint64_t* k1 = S.get<uint64_t>(n);
    uint32_t* v0 = S.get<uint32_t>(n);
    uint32_t* v1 = S.get<uint32_t>(n);
    const int nblocks = (int)blocks_for(n, kRsTile);
    const int64_t hn = 256ll * nblocks;
    uint32_t* hist = S.get<uint32_t>(hn);
    uint32_t* offs = S.get<uint32_t>(hn);
    const int64_t nchunks = (hn + kScanChunk - 1) / kScanChunk;
    uint32_t* sums = S.get<uint32_t>(nchunks);
    int32_t* child = S.get<int32_t>(2 * n);
    int32_t* parent = S.get<int32_t>(2 * n);
    int2* range = S.get<int2>(n);
    int32_t* visits = S.get<int32_t>(n);
    float4* blo = S.get<float4>(n);
    float4* bhi = S.get<float4>(n);
    if (S.err != cudaSuccess) { *msg = "out of device memory (build scratch)"; return SONAR_ERR_OOM; }

    k_morton<<<blocks_for(n, kThreads), kThreads, 0, st>>>(verts, tris, n, d_stats, k0, v0);
    for (int shift = 0; shift < 63; shift += 8) {
        k_rs_hist<<<nblocks, kThreads, 0, st>>>(k0, n, shift, hist, nblocks);
        k_scan_sums<<<(unsigned)nchunks, kThreads, 0, st>>>(hist, hn, sums);
        k_scan_top<<<1, 1024, 0, st>>>(sums, nchunks);
        k_scan_apply<<<(unsigned)nchunks, kThreads, 0, st>>>(hist, hn, sums, offs);
        k_rs_scatter<<<nblocks, kThreads, 0, st>>>(k0, v0, k1, v1, n, shift, offs, nblocks);
        uint64_t* tk = k0; k0 = k1; k1 = tk;
        uint32_t* tv = v0; v0 = v1; v1 = tv;
    }

    // persistent buffers: triangles now, nodes once their count is known
    float4* tri_out = nullptr;
    int32_t* mat_orig = nullptr;
    if (cudaMalloc(&tri_out, sizeof(float4) * 3 * n) != cudaSuccess ||
        cudaMalloc(&mat_orig, sizeof(int32_t) * n) != cudaSuccess) {
        cudaFree(tri_out); cudaFree(mat_orig);
        *msg = "out of device memory (scene)";
        return SONAR_ERR_OOM;
    }
    out->tris = tri_out;
    out->mat_orig = mat_orig;
    out->bytes = sizeof(float4) * 3 * n + sizeof(int32_t) * n;

    k_pack_tris<<<blocks_for(n, kThreads), kThreads, 0, st>>>(verts, tris, mat, v0, n, tri_out, mat_orig);
    int height = 0, depth4 = 0, depth8 = 0;
    if (n <= kLeafMax) {
        out->root = leaf_handle(0, (int32_t)n);
        if (n > 1) {
            k_karras<<<blocks_for(n - 1, kThreads), kThreads, 0, st>>>(k0, n, child, parent, range);
            cudaMemsetAsync(visits, 0, sizeof(int32_t) * (n - 1), st);
            k_refit<<<blocks_for(n, kThreads), kThreads, 0, st>>>(verts, tris, v0, n, child, parent, visits,
                                                                   blo, bhi);
        }
    } else {
        float4* pairs = S.get<float4>(4 * (n - 1));
        CollapseScratch C{};
        C.cost = S.get<float>(8 * n);
        C.dec = S.get<int32_t>(n);
        C.qa = S.get<int32_t>(n);
        C.qb = S.get<int32_t>(n);
        C.picks = S.get<int32_t>(8 * n);
        C.nint = S.get<uint32_t>(n);
        C.prefix = S.get<uint32_t>(n);
        C.fsums = S.get<uint32_t>((n + kScanChunk - 1) / kScanChunk);
        if (S.err != cudaSuccess) { *msg = "out of device memory (build scratch)"; return SONAR_ERR_OOM; }
        k_karras<<<blocks_for(n - 1, kThreads), kThreads, 0, st>>>(k0, n, child, parent, range);
        cudaMemsetAsync(visits, 0, sizeof(int32_t) * (n - 1), st);
        k_refit<<<blocks_for(n, kThreads), kThreads, 0, st>>>(verts, tris, v0, n, child, parent, visits,
                                                               blo, bhi);
        k_pack_nodes<<<blocks_for(n - 1, kThreads), kThreads, 0, st>>>(verts, tris, v0, n, child, range,
                                                                        blo, bhi, pad, pairs);
        float4 root_hi;
        e = cudaMemcpyAsync(&root_hi, bhi, sizeof root_hi, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = collapse_tree<4>(C, n, parent, visits, pairs, st, &out->nodes, &out->n_pairs, &depth4);
        if (e == cudaSuccess)
            e = collapse_tree<8>(C, n, parent, visits, pairs, st, &out->nodes8, &out->n_nodes8, &depth8);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            *msg = std::string("build failed: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? SONAR_ERR_OOM : SONAR_ERR_CUDA;
        }
        memcpy(&height, &root_hi.w, 4);
        out->bytes += sizeof(float4) * (8 * out->n_pairs + 16 * out->n_nodes8);
        out->root = 0;
    }
    out->height = height;
    e = cudaGetLastError();
    if (e != cudaSuccess) { *msg = std::string("build kernel launch failed: ") + cudaGetErrorString(e); return SONAR_ERR_CUDA; }
    // a visit pushes at most W - 1 children, one visit per level of the W-wide
    // tree on any path: the walk never needs more than (W - 1) depth + 1
    // entries.  An 8-wide tree too deep for the stack is dropped (rays then
    // walk the 4-wide one).
    if (3 * depth4 + 1 > kStackMax) {
        *msg = "hierarchy too deep for the traversal stack (4-wide depth " + std::to_string(depth4) + ")";
        return SONAR_ERR_ARG;
    }
    if (out->nodes8 && 7 * depth8 + 1 > kStackMax) {
        cudaFree(out->nodes8);
        out->bytes -= sizeof(float4) * 16 * out->n_nodes8;
        out->nodes8 = nullptr;
        out->n_nodes8 = 0;
    }
    return SONAR_OK;
}

void free_scene(SceneStore* s) {
    cudaFree(s->nodes);
    cudaFree(s->nodes8);
    cudaFree(s->tris);
    cudaFree(s->mat_orig);
    *s = SceneStore{};
}

}  // namespace sonar
