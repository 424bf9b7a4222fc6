// Internal device-side definitions of libsonar (GB300, sm_103a).
//
// Data layout in HBM
//   nodes       4-wide, float4[8] = 128 B (one cache line) per node, per axis
//               two float4 of (lo, hi) plane pairs: [0] (lo.x, hi.x) of children
//               0, 1, [1] of children 2, 3, [2], [3] the same for y, [4], [5] for
//               z, [6] the 4 child handles, [7] unused.  Empty slots: boxes at +inf
//               (never entered), kEmpty.
//   nodes8      8-wide, float4[16] = 256 B per node: two halves in the 4-wide
//               layout, children 0..3 and 4..7.  Built from the same binary
//               hierarchy; a handle >= 0 here indexes nodes8.
//   handles     int32: >= 0 a node index; < 0 a leaf ~((first << 3) | (count - 1)),
//               a run of 1..8 triangles in leaf order; kEmpty an empty slot.
//   triangles   float4[3] per triangle in leaf order (48 B):
//               (v0, material id bits), (v1, caller's index bits), (v2, 0).
//   polar       [n_range_bins][n_az_bins] f32 per sensor (row = range bin).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sonar.h"

namespace sonar {

constexpr int kLeafMax = 2;          // triangles per collapsed leaf (a heightfield cell; 4 tested 7 % slower)
constexpr int kStackMax = 96;        // traversal stack entries (tree height is checked at build)
constexpr int32_t kEmpty = (int32_t)0x80000000;
constexpr int kMaxMat = 1024;
constexpr int kMaxCols = 64;         // azimuth columns per binning unit, at most
constexpr uint32_t kNoKey = 0xFFFFFFFFu;

__host__ __device__ inline int32_t leaf_handle(int32_t first, int32_t count) {
    return ~((first << 3) | (count - 1));
}

// The scene as the kernels see it.
struct SceneDev {
    const float4* nodes;      // [n_nodes * 8], 4-wide
    const float4* tris;       // [n_tris * 3]
    const int32_t* mat_orig;  // [n_tris] material of the caller's triangle index
    int32_t root;             // root handle (kEmpty if the scene has no triangles), both trees
    int32_t n_tris;
    const float4* nodes8;     // [n_nodes8 * 16], 8-wide, or null (none built)
};

// SensorDev::occ, the ray-cast variant: bit kTraceCap caps registers at 64 so
// that 32 one-warp blocks fit an SM; bit kTraceWide walks the 8-wide tree.
constexpr int kTraceCap = 8;
constexpr int kTraceWide = 16;

// One sensor of a render, with everything the kernels derive from it.
struct SensorDev {
    float pos[3];
    float rot[9];
    int32_t nb, ne, nr, naz;
    float hfov, vfov, rmin, rmax;
    float inv_dr;        // n_range_bins / (r_max - r_min)
    float fan_scale;     // fan pixels per metre
    int32_t fan_w, fan_h;
    uint32_t seed_lo, seed_hi, frame_lo, frame_hi;
    int32_t scene;       // index into the scene table
    int32_t cols;        // binning: azimuth columns per work unit
    int32_t n_tiles;     // binning work units of this sensor = ceil(naz / cols)
    int32_t tb;          // trace: beams per warp tile (elevations = 32 / tb)
    int32_t occ;         // trace: variant bits kTraceCap, kTraceWide
    int32_t trace_blocks;  // trace: one-warp blocks covering the sensor
    int32_t fold_beams;  // binning: deterministic fold into per-beam rows (fits in shared memory)
    int64_t polar_off, hits_off, fan_off, rowmax_off;
    float4* trig;        // float-float sin/cos of the beam azimuths [nb] and elevations [ne]
    uint4* fan_lut;      // per-pixel fan coordinates shared with same-geometry sensors (nullptr: compute)
    uint32_t* trig_stamp;  // batch: per k_trig block, the trig_version its table entries were built for
    uint32_t trig_version; // batch: bumped whenever an update changes the fields of view
    uint32_t* fan_stamp;   // table owners: per table block, the fan_version it was last built for
    uint32_t fan_version;  // table owners: bumped whenever an update changes the fan geometry
    uint32_t pad_;
};

// A work unit: the azimuth columns [c0, c1) of one sensor, i.e. every ray
// of the beams that fall into those columns.
struct Unit {
    int32_t sensor;
    int32_t c0, c1;
    int32_t rays;     // host: orders the work list
    int32_t scene;    // the sensor's scene (its descriptor is fetched beside the sensor's)
};

// First beam whose azimuth bin floor((2i+1) naz / (2 nb)) is >= c.
__host__ __device__ inline int32_t first_beam_of_col(int64_t c, int64_t nb, int64_t naz) {
    // (2i + 1) naz >= 2 nb c  <=>  i >= (2 nb c - naz) / (2 naz)
    const int64_t num = 2 * nb * c - naz;
    if (num <= 0) return 0;
    const int64_t den = 2 * naz;
    const int64_t i = (num + den - 1) / den;
    return (int32_t)(i < nb ? i : nb);
}

// ---- order-preserving float <-> uint32 encoding (for atomicMax on floats) ----
__device__ __forceinline__ uint32_t ord_enc(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(uint32_t e) {
    return __uint_as_float((e & 0x80000000u) ? (e & 0x7FFFFFFFu) : ~e);
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----
// Round: multiply words 0 and 2 by the two round multipliers (full 64-bit
// products); the new words are (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2),
// hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)); the key advances by the Weyl increments
// between rounds.
struct U4 { uint32_t x, y, z, w; };

// The ten round keys of one Philox key (k_r = k + r * Weyl increment),
// computed once per key so that a round is two wide multiplies and two XORs.
struct PhiloxKey {
    uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKey philox_key(uint32_t lo, uint32_t hi) {
    PhiloxKey K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = lo + (uint32_t)r * 0x9E3779B9u;
        K.k1[r] = hi + (uint32_t)r * 0xBB67AE85u;
        // opaque to the compiler: kept in registers rather than recomputed per use
        asm volatile("" : "+r"(K.k0[r]), "+r"(K.k1[r]));
    }
    return K;
}
__device__ __forceinline__ U4 philox10(U4 c, const PhiloxKey& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = U4{(uint32_t)(p1 >> 32) ^ c.y ^ K.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[r],
               (uint32_t)p0};
    }
    return c;
}
__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) { return philox10(c, philox_key(k0, k1)); }

// -2 ln u for u = (x + 1) / 2^32, without branches.  With u = 2^e f and f in
// [sqrt(1/2), sqrt(2)), ln u = e ln 2 + 2 atanh(z), z = (f - 1) / (f + 1),
// |z| <= 3 - 2 sqrt(2) < 0.1716, and 2 atanh(z) = 2 z (1 + z^2/3 + ... +
// z^10/11) to well below FP32 rounding (the next term is < 2^-33 relative).
// For u >= sqrt(1/2) (e = 0), f - 1 = -(2^32 - 1 - x) / 2^32 is taken from the
// integer complement, so u close to 1 keeps its relative accuracy.
__device__ __forceinline__ float neg2log_u(uint32_t x) {
    const bool upper = x >= 0xB504F333u;   // (x + 1) / 2^32 >= sqrt(1/2)
    const float u = fmaf((float)x, 0x1p-32f, 0x1p-32f);
    const uint32_t bits = __float_as_uint(u);
    float f = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);   // mantissa in [1, 2)
    int e = (int)(bits >> 23) - 127;
    const bool fold = f > 1.41421356f;
    f = fold ? 0.5f * f : f;
    e = fold ? e + 1 : e;
    float d = f - 1.0f;                                                // exact
    d = upper ? -(float)(0xFFFFFFFFu - x) * 0x1p-32f : d;
    e = upper ? 0 : e;
    const float z = __fdividef(d, 2.0f + d);
    const float z2 = z * z;
    float p = fmaf(z2, 1.0f / 11.0f, 1.0f / 9.0f);
    p = fmaf(z2, p, 1.0f / 7.0f);
    p = fmaf(z2, p, 1.0f / 5.0f);
    p = fmaf(z2, p, 1.0f / 3.0f);
    p = fmaf(z2, p, 1.0f);
    // e in [-32, 0]: exact as a float without a conversion instruction
    const float ef = __uint_as_float(0x4B000000u | (uint32_t)(e + 64)) - 8388672.0f;
    return -2.0f * fmaf(ef, 0.693147180559945f, 2.0f * z * p);
}

// sqrt(v) for v >= 0 from the reciprocal square root (a few ulp).
__device__ __forceinline__ float sqrt_nonneg(float v) { return v > 0.0f ? v * rsqrtf(v) : 0.0f; }

// The two noise streams of a frame (Eq. 4 and 5), key = seed.  Additive term:
// Rayleigh(sigma_sa) by inversion of word (bin mod 4) of counter (bin / 4,
// frame lo, 1, frame hi), so that four neighbouring bins share one Philox
// block.  Multiplicative term: the cosine branch of Box-Muller for N(0,
// sigma_sm) on words 1, 2 of counter (bin, frame lo, 0, frame hi) (words 0
// and 3 unused).  Counter word 2 tells the streams apart.
__device__ __forceinline__ U4 additive_words(uint32_t quad, uint32_t frame_lo, uint32_t frame_hi,
                                             const PhiloxKey& K) {
    return philox10(U4{quad, frame_lo, 1u, frame_hi}, K);
}
__device__ __forceinline__ U4 bin_draws(uint32_t bin, const SensorDev& s, const PhiloxKey& K) {
    return philox10(U4{bin, s.frame_lo, 0u, s.frame_hi}, K);
}
__device__ __forceinline__ uint32_t word_of(const U4& x, uint32_t j) {
    return j == 0 ? x.x : j == 1 ? x.y : j == 2 ? x.z : x.w;
}
__device__ __forceinline__ float rayleigh_of(uint32_t word, float sigma_sa) {
    return sigma_sa * sqrt_nonneg(neg2log_u(word));
}
__device__ __forceinline__ float gauss_of(const U4& x, float sigma_sm) {
    const float u2 = fmaf((float)x.z, 0x1p-32f, 0x1p-32f);
    return sigma_sm * sqrt_nonneg(neg2log_u(x.y)) * cospif(2.0f * u2);
}
__device__ __forceinline__ float w_sm_of(uint32_t bin, const SensorDev& s, float sigma_sm, const PhiloxKey& K) {
    return gauss_of(bin_draws(bin, s, K), sigma_sm);
}

// Copies a descriptor word by word with the lanes of one warp (lane < 32).
template <class T>
__device__ __forceinline__ void copy_words(T* dst, const T* src, int lane) {
    static_assert(sizeof(T) % 4 == 0, "descriptor of whole words");
    for (int i = lane; i < (int)(sizeof(T) / 4); i += 32)
        reinterpret_cast<uint32_t*>(dst)[i] = __ldg(reinterpret_cast<const uint32_t*>(src) + i);
}

// ---- kernel argument blocks ----

struct TraceCounters {
    unsigned long long* visits;     // node-pair visits
    unsigned long long* tests;      // triangle tests
    unsigned long long* exact;      // tests resolved in FP64
    uint32_t* node_bits;            // touched node pairs (bitmap)
    uint32_t* tri_bits;             // touched triangles (bitmap)
};

// Ray casting: one-warp blocks of 32 rays.
struct TraceArgs {
    const SensorDev* sensors;   // batch: device array; single: nullptr (use `one`)
    const SceneDev* scenes;     // batch: device table; single: nullptr (use `one_scene`)
    const int4* block_map;      // batch: per block (sensor, tile of that sensor, its scene, 0)
    int32_t n_sensors;
    SensorDev one;
    SceneDev one_scene;
    sonar_params params;
    sonar_hit* hits;            // written unless counting (the caller's buffer or scratch)
    uint32_t* err;
    TraceCounters tc;           // counting launches only
    int32_t* zero_word;         // cleared for the launch after this one (a work counter), or nullptr
};

// Binning and noise over column-tile work units.
struct BinArgs {
    const SensorDev* sensors;   // batch: device array; single: nullptr (use `one`)
    const Unit* units;          // batch: device work list; single: nullptr
    const SceneDev* scenes;     // batch: device table; single: nullptr (use `one_scene`)
    int32_t* work_counter;      // persistent work list counter (nullptr: unit = blockIdx.x)
    int32_t n_units;
    int32_t n_mat;
    SensorDev one;
    SceneDev one_scene;
    const float* theta;         // (alpha, gain, mu[...])
    sonar_params params;
    const sonar_hit* hits;      // the trace kernel's records
    float* noised;
    float* binned;
    uint32_t* rowmax;           // normalise = 2: ordered-encoded image maximum per sensor
    uint32_t* err;
};

// Normalisation: one warp per (sensor, range row).
struct NormArgs {
    const SensorDev* sensors;   // batch: device array; single: nullptr (use `one`)
    const int32_t* row_map;     // batch: sensor of each row
    int32_t n_sensors;
    int64_t total_rows;         // sum of n_range_bins over the sensors
    SensorDev one;
    const float* noised;
    const uint32_t* gmax;       // normalise = 2: ordered-encoded image maximum at rowmax_off
    int32_t normalise;
    float* polar;
};

constexpr int kFanTile = 4096;  // pixels per coordinate-table block
constexpr int kFanSide = 64;    // resample blocks are kFanSide x kFanSide pixel squares (compact in polar)
// Square resample blocks of a w x h fan image.
__host__ __device__ inline int32_t fan_squares(int32_t w, int32_t h) {
    return ((w + kFanSide - 1) / kFanSide) * ((h + kFanSide - 1) / kFanSide);
}
// The fan of a sensor that shares no coordinate table (single frames, sensors
// of unique geometry) goes in smaller squares: one frame's fan is then several
// blocks per SM instead of about one.
constexpr int kTileSide = 32;
__host__ __device__ inline int32_t tile_squares(int32_t w, int32_t h) {
    return ((w + kTileSide - 1) / kTileSide) * ((h + kTileSide - 1) / kTileSide);
}

// DVL measurement of n poses (four beams each).
struct DvlArgs {
    SceneDev scene;
    const float* pose;        // [n][12]: position, sensor->world rotation (row-major)
    const float* vel_world;   // [n][3]
    int64_t n;
    float beam[4][3];         // sensor-frame unit beams (from the tilt, in FP64 on the host)
    float r_min, r_max, sigma_b, t0, t1, t_lost;
    int32_t min_beams;
    uint32_t seed_lo, seed_hi;
    float* ranges;            // [n][4] out
    float* vel;               // [n][3] out
    int32_t* flags;           // [n] out
    float* period;            // [n] out
    uint32_t* err;
};

// Underwater image formation coefficients (Eq. 1), per colour channel R, G, B.
struct UwCoef {
    float b_attn[3];   // attenuation
    float b_bs[3];     // backscatter
    float b_inf[3];    // veiling light
};

// Fan resample: kFanSide x kFanSide pixel squares of one sensor, reading the normalised image.
struct FanArgs {
    const SensorDev* sensors;   // batch: device array; single: nullptr
    const int2* block_map;      // batch: per block (sensor, block of that sensor); single: nullptr
    int32_t n_sensors;
    SensorDev one;
    const float* polar;
    float* fan;
};

// Fan of the users of a shared coordinate table: per block (owner, block of
// its pixels, users members[m0 .. m1)); one thread serves up to kFanGroup frames.
constexpr int kFanGroup = 2;     // frames per grouped fan block (more frames per thread evict lines that neighbouring pixels reuse)
struct FanGroupArgs {
    const SensorDev* sensors;
    const int4* block_map;
    const int32_t* members;
    const float* polar;
    float* fan;
};

// Fan coordinate tables: per table block (owner sensor, block of its pixels).
struct FanLutArgs {
    const SensorDev* sensors;
    const int2* block_map;
    uint4* const* luts;         // per owner sensor: its table
};

// A work unit of the adjoint: canonical rays [r0, r1) of one sensor.
struct AdjUnit {
    int32_t sensor, r0, r1, scene;
};

struct RowInfo {
    float m;        // group maximum of I~ (normalise mode 1: per row; mode 2: whole image)
    float c;        // sum_k G_k I~_k / m^2
    int32_t arg;    // bin index of the maximum (lowest on ties) within the sensor image
    int32_t valid;  // m > 0
};

struct AdjArgs {
    const SensorDev* sensors;
    const AdjUnit* units;       // batch: device work list; single: nullptr (chunks of `chunk` rays)
    const SceneDev* scenes;
    int32_t* work_counter;      // persistent work list counter (nullptr: unit = blockIdx.x)
    int32_t n_units;
    int32_t n_mat;
    int32_t chunk;
    SensorDev one;
    SceneDev one_scene;
    const float* theta;
    sonar_params params;
    const float* grad;          // dL/dN, packed like the polar output
    const sonar_hit* hits;      // the hit records (stored, or recomputed just before)
    const RowInfo* rowinfo;     // per sensor: at rowmax_off
    double* partials;           // [n_units][2 + n_mat]
    uint32_t* err;
};

}  // namespace sonar
