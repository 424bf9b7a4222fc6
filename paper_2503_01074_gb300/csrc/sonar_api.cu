// C ABI of libsonar: contexts, scenes, single-frame and batched rendering,
// the adjoint, the autotuner and the counter mode.  Host code only; kernels
// live in bvh_build.cu, trace.cu, render.cu, image.cu and dvl.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sonar_host.h"
#include "sonar_internal.cuh"

using namespace sonar;

namespace {

struct Tune {
    int cols = 0;     // binning: azimuth columns per work unit (0: derive)
    int tb = 0;       // tracing: beams per warp tile, elevations = 32 / tb (0: derive)
    int block = 128;  // binning: threads per block
    int occ = 0;      // tracing variant: kTraceCap caps registers at 64 (32 one-warp blocks per SM),
                      // kTraceWide walks the 8-wide tree
};

using ShapeKey = std::array<int, 4>;   // n_beams, n_elev, n_range_bins, n_az_bins

// A device buffer that grows on demand (stream-ordered allocation).
struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct sonar_ctx {
    int device = 0;
    int sm_count = 1;
    std::vector<SceneStore> scenes;
    std::vector<bool> alive;
    std::string last_error;
    uint32_t* d_err = nullptr;
    Scratch rowmax, noised, rowinfo, partials, counters, hits, trig;
    // the exact-ray tables last built by a single-sensor call: their buffer and
    // the angular geometry they hold (beams, elevations, fields of view)
    const float4* trig_at = nullptr;
    int trig_nb = 0, trig_ne = 0;
    float trig_hfov = 0.0f, trig_vfov = 0.0f;
    std::map<ShapeKey, Tune> tune;
};

struct sonar_batch;

namespace {

sonar_status fail(sonar_ctx* ctx, sonar_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

sonar_status cuda_fail(sonar_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? SONAR_ERR_OOM : SONAR_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

cudaError_t grow(Scratch& s, size_t bytes, cudaStream_t st) {
    if (s.bytes >= bytes && s.p) return cudaSuccess;
    if (s.p) cudaFreeAsync(s.p, st);
    s.p = nullptr;
    s.bytes = 0;
    size_t want = std::max(bytes, (size_t)256);
    cudaError_t e = cudaMallocAsync(&s.p, want, st);
    if (e == cudaSuccess) s.bytes = want;
    return e;
}

bool finite_f(float x) { return std::isfinite(x); }

sonar_status check_sensor(sonar_ctx* ctx, const sonar_sensor* s) {
    if (!s) return fail(ctx, SONAR_ERR_ARG, "sensor is NULL");
    if (s->n_beams < 1 || s->n_elev < 1 || s->n_range_bins < 1 || s->n_az_bins < 1)
        return fail(ctx, SONAR_ERR_ARG, "sensor counts must be >= 1");
    if ((int64_t)s->n_beams * s->n_elev > 0x7FFFFFFFll)
        return fail(ctx, SONAR_ERR_ARG, "n_beams * n_elev exceeds 2^31 - 1");
    if ((int64_t)s->n_range_bins * s->n_az_bins > 0x7FFFFFFEll)
        return fail(ctx, SONAR_ERR_ARG, "n_range_bins * n_az_bins exceeds 2^31 - 2");
    for (int k = 0; k < 3; ++k)
        if (!finite_f(s->pos[k])) return fail(ctx, SONAR_ERR_ARG, "sensor position not finite");
    for (int k = 0; k < 9; ++k)
        if (!finite_f(s->rot[k])) return fail(ctx, SONAR_ERR_ARG, "sensor rotation not finite");
    const float pi = 3.14159265358979f;
    if (!(s->hfov > 0.0f && s->hfov <= pi)) return fail(ctx, SONAR_ERR_ARG, "hfov must be in (0, pi]");
    if (!(s->vfov > 0.0f && s->vfov <= pi)) return fail(ctx, SONAR_ERR_ARG, "vfov must be in (0, pi]");
    if (!(s->r_min >= 0.0f && s->r_max > s->r_min && finite_f(s->r_max)))
        return fail(ctx, SONAR_ERR_ARG, "need 0 <= r_min < r_max < inf");
    return SONAR_OK;
}

sonar_status check_params(sonar_ctx* ctx, const sonar_params* p) {
    if (!p) return fail(ctx, SONAR_ERR_ARG, "params is NULL");
    if (!(p->sigma_sa >= 0.0f && finite_f(p->sigma_sa))) return fail(ctx, SONAR_ERR_ARG, "sigma_sa must be >= 0");
    if (!(p->sigma_sm >= 0.0f && finite_f(p->sigma_sm))) return fail(ctx, SONAR_ERR_ARG, "sigma_sm must be >= 0");
    if (!(p->sigma_phi > 0.0f && finite_f(p->sigma_phi))) return fail(ctx, SONAR_ERR_ARG, "sigma_phi must be > 0");
    if (p->normalise < 0 || p->normalise > 2) return fail(ctx, SONAR_ERR_ARG, "normalise must be 0, 1 or 2");
    if (p->two_sided < 0 || p->two_sided > 1) return fail(ctx, SONAR_ERR_ARG, "two_sided must be 0 or 1");
    if (p->clip_tmax < 0 || p->clip_tmax > 1) return fail(ctx, SONAR_ERR_ARG, "clip_tmax must be 0 or 1");
    if (p->accumulate < 0 || p->accumulate > 1) return fail(ctx, SONAR_ERR_ARG, "accumulate must be 0 or 1");
    return SONAR_OK;
}

sonar_status check_scene(sonar_ctx* ctx, int32_t id) {
    if (id < 0 || id >= (int32_t)ctx->scenes.size() || !ctx->alive[id])
        return fail(ctx, SONAR_ERR_ARG, "unknown scene id " + std::to_string(id));
    return SONAR_OK;
}

sonar_status check_nmat(sonar_ctx* ctx, int32_t scene, int32_t n_mat) {
    if (n_mat < 1 || n_mat > kMaxMat) return fail(ctx, SONAR_ERR_ARG, "n_mat must be in [1, 1024]");
    if (ctx->scenes[scene].max_mat >= n_mat)
        return fail(ctx, SONAR_ERR_ARG, "scene uses material id " + std::to_string(ctx->scenes[scene].max_mat) +
                                             " >= n_mat " + std::to_string(n_mat));
    return SONAR_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Tile shape for a sensor: the tuning cache entry, else one block-wide ray
// tile per unit, bounded by the shared-memory column block.
Tune tune_for(const sonar_ctx* ctx, const sonar_sensor& s) {
    Tune t;
    auto it = ctx->tune.find(ShapeKey{s.n_beams, s.n_elev, s.n_range_bins, s.n_az_bins});
    if (it != ctx->tune.end()) t = it->second;
    const int bpc = std::max(1, s.n_beams / std::max(1, s.n_az_bins));
    if (t.cols <= 0) t.cols = std::max(1, t.block / std::max(1, s.n_elev * bpc));
    // a unit's column block, its bitmap (a bit per bin) and its list (at most a
    // word per bin) fit the dynamic shared memory: bins * 65 / 32 words
    const int max_cols_smem = std::max(1, (int)(kMaxDynSmem / 4 * 32 / 65) / s.n_range_bins);
    t.cols = std::max(1, std::min({t.cols, s.n_az_bins, max_cols_smem, kMaxCols}));
    if (t.block < 32 || t.block > 512 || (t.block & 31)) t.block = 128;
    if (t.tb <= 0) t.tb = 8;
    if (t.tb > 32 || (t.tb & (t.tb - 1))) t.tb = 8;
    return t;
}

// The tree a ray-cast launch of `blocks` one-warp blocks walks: the 8-wide one
// when the launch is at most one wave (32 resident blocks per SM), where a
// ray's chain of dependent node loads sets the time, else the 4-wide one,
// which costs fewer instructions per ray once the SMs have warps to switch to.
int wide_for_launch(const sonar_ctx* ctx, int64_t blocks) {
    return blocks <= 32ll * ctx->sm_count ? kTraceWide : 0;
}

// The ray-cast variant of one sensor's own launch (tile tb from its tuning
// row, variant `occ` of that row): the tree by the launch size, and no
// register cap for a launch of at most one wave, which cannot use the
// occupancy that the cap buys.
int single_variant(const sonar_ctx* ctx, const sonar_sensor& s, int tb, int occ) {
    const int64_t be = 32 / tb;
    const int64_t blocks = ((s.n_beams + tb - 1) / tb) * ((s.n_elev + be - 1) / be);
    if (wide_for_launch(ctx, blocks)) return kTraceWide;
    return occ & ~kTraceWide;
}

// A single frame alone on the GPU: the tuned shapes, but binning units of
// about two per SM (the batch tunes may favour few, large units) and at least
// four columns wide, a multiple of 4 where the row allows, so that the noise
// pass draws four bins per Philox block; and the ray-cast variant chosen by the
// frame's own launch size.
Tune single_tune(const sonar_ctx* ctx, const sonar_sensor& s) {
    Tune t = tune_for(ctx, s);
    int cols = std::max(4, s.n_az_bins / (2 * ctx->sm_count));
    if (s.n_az_bins % 4 == 0) cols &= ~3;
    const int max_cols_smem = std::max(1, (int)(kMaxDynSmem / 4 * 32 / 65) / s.n_range_bins);
    t.cols = std::max(1, std::min({cols, s.n_az_bins, max_cols_smem, kMaxCols}));
    t.occ = single_variant(ctx, s, t.tb, t.occ);
    return t;
}

// Most beams a binning unit of this sensor covers (its columns' beams).
int64_t unit_beams_max(const SensorDev& s) {
    int64_t most = 0;
    for (int t = 0; t < s.n_tiles; ++t) {
        const int64_t c0 = (int64_t)t * s.cols, c1 = std::min<int64_t>(c0 + s.cols, s.naz);
        most = std::max<int64_t>(most, first_beam_of_col(c1, s.nb, s.naz) - first_beam_of_col(c0, s.nb, s.naz));
    }
    return most;
}
int64_t unit_rays_max(const SensorDev& s) { return unit_beams_max(s) * (int64_t)s.ne; }

SensorDev make_sensor(const sonar_sensor& s, uint64_t seed, uint64_t frame, const Tune& t, int fan_w,
                      int fan_h) {
    SensorDev d{};
    memcpy(d.pos, s.pos, sizeof d.pos);
    memcpy(d.rot, s.rot, sizeof d.rot);
    d.nb = s.n_beams;
    d.ne = s.n_elev;
    d.nr = s.n_range_bins;
    d.naz = s.n_az_bins;
    d.hfov = s.hfov;
    d.vfov = s.vfov;
    d.rmin = s.r_min;
    d.rmax = s.r_max;
    d.inv_dr = (float)((double)s.n_range_bins / ((double)s.r_max - (double)s.r_min));
    d.fan_w = fan_w;
    d.fan_h = fan_h;
    if (fan_w > 0 && fan_h > 0) {
        const double sx = fan_w / (2.0 * (double)s.r_max * std::sin((double)s.hfov / 2.0));
        const double sy = fan_h / (double)s.r_max;
        d.fan_scale = (float)std::min(sx, sy);
    }
    d.seed_lo = (uint32_t)seed;
    d.seed_hi = (uint32_t)(seed >> 32);
    d.frame_lo = (uint32_t)frame;
    d.frame_hi = (uint32_t)(frame >> 32);
    d.cols = t.cols;
    d.n_tiles = (s.n_az_bins + t.cols - 1) / t.cols;
    const int tb = (t.tb >= 1 && t.tb <= 32 && (t.tb & (t.tb - 1)) == 0) ? t.tb : 8;   // beams per warp tile
    d.tb = tb;
    d.occ = t.occ;
    const int64_t be = 32 / tb;   // ray-cast blocks: one warp on tb beams x be elevations
    d.trace_blocks = (int32_t)(((s.n_beams + tb - 1) / tb) * ((s.n_elev + be - 1) / be));
    // The per-beam fold when columns hold several beams (n_beams > n_az_bins:
    // with one beam per column both folds add in the same order, and the
    // all-warp fold is faster) and its rows fit in shared memory next to the
    // column block and the list.  The choice depends on the sensor shape alone
    // (it is made for one column per unit), so every tile shape folds in the
    // same order; wider units are narrowed until they fit.
    auto fits = [&](const SensorDev& x) {
        const int64_t bins = (int64_t)x.nr * x.cols;
        const int64_t need = bins + unit_beams_max(x) * x.nr + (bins + 31) / 32 + std::min<int64_t>(unit_rays_max(x), bins);
        return need * (int64_t)sizeof(float) <= (int64_t)kMaxDynSmem;
    };
    SensorDev one_col = d;
    one_col.cols = 1;
    one_col.n_tiles = s.n_az_bins;
    d.fold_beams = (s.n_beams > s.n_az_bins && fits(one_col)) ? 1 : 0;
    while (d.fold_beams && d.cols > 1 && !fits(d)) {
        d.cols = std::max(1, d.cols / 2);
        d.n_tiles = (s.n_az_bins + d.cols - 1) / d.cols;
    }
    return d;
}

}  // namespace

// ===========================================================================
// context
// ===========================================================================

extern "C" const char* sonar_version(void) {
    return "libsonar 1.0 (sm_103a; 4-wide LBVH + certified FP32 Moller-Trumbore with float-float exact decisions; Philox4x32-10)";
}

extern "C" sonar_status sonar_create(int32_t device, sonar_ctx_t* out) {
    if (!out) return SONAR_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SONAR_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SONAR_ERR_CUDA;
    sonar_ctx* ctx = new sonar_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(uint32_t)) != cudaSuccess) {
        delete ctx;
        return SONAR_ERR_OOM;
    }
    set_kernel_attributes();
    cudaGetLastError();
    *out = ctx;
    return SONAR_OK;
}

extern "C" sonar_status sonar_destroy(sonar_ctx_t ctx) {
    if (!ctx) return SONAR_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& s : ctx->scenes) free_scene(&s);
    for (Scratch* s : {&ctx->rowmax, &ctx->noised, &ctx->rowinfo, &ctx->partials, &ctx->counters, &ctx->hits,
                       &ctx->trig})
        if (s->p) cudaFreeAsync(s->p, 0);
    cudaDeviceSynchronize();
    cudaFree(ctx->d_err);
    delete ctx;
    return SONAR_OK;
}

extern "C" const char* sonar_last_error(sonar_ctx_t ctx) {
    return ctx ? ctx->last_error.c_str() : "";
}

extern "C" sonar_status sonar_check(sonar_ctx_t ctx, uint32_t* bits) {
    if (!ctx) return SONAR_ERR_ARG;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    CU(cudaDeviceSynchronize(), "device synchronisation");
    uint32_t w = 0;
    CU(cudaMemcpy(&w, ctx->d_err, sizeof w, cudaMemcpyDeviceToHost), "reading the error word");
    if (bits) *bits = w;
    if (w) {
        CU(cudaMemset(ctx->d_err, 0, sizeof(uint32_t)), "clearing the error word");
        return fail(ctx, SONAR_ERR_DEVICE, "device error word 0x" + std::to_string(w));
    }
    return SONAR_OK;
}

// ===========================================================================
// scenes
// ===========================================================================

extern "C" sonar_status sonar_scene_upload(sonar_ctx_t ctx, const float* d_verts, int64_t n_verts,
                                           const int32_t* d_tris, const int32_t* d_mat, int64_t n_tris,
                                           void* stream, int32_t* scene_id) {
    if (!ctx || !scene_id) return fail(ctx, SONAR_ERR_ARG, "NULL context or scene_id");
    if (n_tris < 0 || n_verts < 0) return fail(ctx, SONAR_ERR_ARG, "negative counts");
    if (n_tris >= (1ll << 28) - 2) return fail(ctx, SONAR_ERR_ARG, "n_tris must be < 2^28 - 2");
    if (n_verts >= (1ll << 31)) return fail(ctx, SONAR_ERR_ARG, "n_verts must be < 2^31");
    if (n_tris > 0 && (!d_verts || !d_tris || !d_mat || n_verts == 0))
        return fail(ctx, SONAR_ERR_ARG, "NULL scene arrays");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    SceneStore s;
    std::string msg;
    const sonar_status st = build_scene(d_verts, n_verts, d_tris, d_mat, n_tris, (cudaStream_t)stream, &s, &msg);
    if (st != SONAR_OK) {
        free_scene(&s);
        return fail(ctx, st, msg);
    }
    ctx->scenes.push_back(s);
    ctx->alive.push_back(true);
    *scene_id = (int32_t)ctx->scenes.size() - 1;
    return SONAR_OK;
}

extern "C" sonar_status sonar_scene_release(sonar_ctx_t ctx, int32_t id) {
    if (!ctx) return SONAR_ERR_ARG;
    sonar_status st = check_scene(ctx, id);
    if (st) return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    CU(cudaDeviceSynchronize(), "device synchronisation");
    free_scene(&ctx->scenes[id]);
    ctx->alive[id] = false;
    return SONAR_OK;
}

extern "C" sonar_status sonar_scene_info(sonar_ctx_t ctx, int32_t id, int64_t out[5]) {
    if (!ctx || !out) return fail(ctx, SONAR_ERR_ARG, "NULL argument");
    sonar_status st = check_scene(ctx, id);
    if (st) return st;
    const SceneStore& s = ctx->scenes[id];
    out[0] = s.n_tris;
    out[1] = s.n_pairs;
    out[2] = s.height;
    out[3] = s.max_mat;
    out[4] = (int64_t)s.bytes;
    return SONAR_OK;
}

// ===========================================================================
// single-frame rendering
// ===========================================================================

namespace {


// Shared memory of a binning block: the column block of the unit, the per-beam
// rows of the fold if any, a bitmap of the bins with returns, and the list of
// those bins (no more entries than rays, nor than bins).
size_t bin_smem(const SensorDev& s) {
    const int64_t bins = (int64_t)s.nr * s.cols;
    const int64_t beams = s.fold_beams ? unit_beams_max(s) * s.nr : 0;   // per-beam rows of the fold
    return (size_t)(bins + beams + (bins + 31) / 32 + std::min<int64_t>(unit_rays_max(s), bins)) * sizeof(float);
}

// The context's exact-ray table buffer, grown to `entries`; a new buffer holds
// no tables yet.
cudaError_t grow_trig(sonar_ctx* ctx, size_t entries, cudaStream_t s) {
    const void* before = ctx->trig.p;
    const cudaError_t e = grow(ctx->trig, sizeof(float4) * entries, s);
    if (e != cudaSuccess || ctx->trig.p != before || ctx->trig.bytes < sizeof(float4) * entries) ctx->trig_at = nullptr;
    return e;
}

// The exact-ray tables of one sensor's call.  They depend on the angular
// geometry only, so a call with the same geometry and table buffer as the last
// build skips the launch (calls on a context are stream-ordered); while the
// stream is being captured into a graph the launch is always recorded, so that
// a replay rebuilds the tables it reads.
cudaError_t single_trig(sonar_ctx* ctx, const SensorDev& S, cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone && ctx->trig_at == S.trig && ctx->trig_nb == S.nb && ctx->trig_ne == S.ne &&
        ctx->trig_hfov == S.hfov && ctx->trig_vfov == S.vfov)
        return cudaSuccess;
    e = launch_trig(nullptr, S, 1, S.nb + S.ne, s);
    const bool keep = e == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    ctx->trig_at = keep ? S.trig : nullptr;
    ctx->trig_nb = S.nb;
    ctx->trig_ne = S.ne;
    ctx->trig_hfov = S.hfov;
    ctx->trig_vfov = S.vfov;
    return e;
}

// Trace, bin and noise of one sensor (polar_off = hits_off = rowmax_off = 0).
sonar_status single_forward(sonar_ctx* ctx, const SensorDev& S, const SceneDev& sc, const sonar_params* p,
                            const float* d_theta, int32_t n_mat, sonar_hit* hits, float* noised, float* binned,
                            uint32_t* gmax, int block, cudaStream_t s) {
    if (p->normalise == 2) CU(cudaMemsetAsync(gmax, 0, sizeof(uint32_t), s), "cudaMemsetAsync");
    CU(single_trig(ctx, S, s), "trig launch");
    TraceArgs t{};
    t.one = S;
    t.one_scene = sc;
    t.params = *p;
    t.hits = hits;
    t.err = ctx->d_err;
    CU(launch_trace(t, S.trace_blocks, S.occ, s), "trace launch");
    BinArgs a{};
    a.n_units = S.n_tiles;
    a.n_mat = n_mat;
    a.one = S;
    a.one_scene = sc;
    a.theta = d_theta;
    a.params = *p;
    a.hits = hits;
    a.noised = noised;
    a.binned = binned;
    a.rowmax = gmax;
    a.err = ctx->d_err;
    CU(launch_bin(a, p->accumulate == 0, S.n_tiles, block, bin_smem(S), s), "binning launch");
    return SONAR_OK;
}

// Normalisation and fan of one sensor (polar_off = fan_off = rowmax_off = 0).
sonar_status single_post(sonar_ctx* ctx, const SensorDev& S, int normalise, const float* noised,
                         const uint32_t* gmax, float* polar, float* fan, cudaStream_t s) {
    NormArgs n{};
    n.one = S;
    n.total_rows = S.nr;
    n.noised = noised;
    n.gmax = gmax;
    n.normalise = normalise;
    n.polar = polar;
    CU(launch_norm(n, s), "normalisation launch");
    if (fan) {
        FanArgs f{};
        f.one = S;
        f.polar = polar;
        f.fan = fan;
        CU(launch_fan_tiles(f, tile_squares(S.fan_w, S.fan_h), s), "fan launch");
    }
    return SONAR_OK;
}

// Rays per adjoint work unit: about four units per SM over the whole render,
// a multiple of the block size.
int adj_chunk(int64_t rays, int sm_count, int block) {
    // about 16 units per SM: the per-ray gather is latency-bound and wants
    // many resident blocks
    int64_t c = rays / (16 * (int64_t)sm_count);
    c = (c + block - 1) / block * block;
    return (int)std::max<int64_t>(block, std::min<int64_t>(c, 64ll * block));
}

}  // namespace

extern "C" sonar_status sonar_render(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                                     const sonar_params* params, const float* d_theta, int32_t n_mat,
                                     uint64_t seed, uint64_t frame, const sonar_outputs* out,
                                     void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    sonar_status st;
    if ((st = check_scene(ctx, scene_id)) || (st = check_sensor(ctx, sensor)) || (st = check_params(ctx, params)) ||
        (st = check_nmat(ctx, scene_id, n_mat)))
        return st;
    if (!d_theta) return fail(ctx, SONAR_ERR_ARG, "d_theta is NULL");
    if (!out || !out->polar) return fail(ctx, SONAR_ERR_ARG, "outputs or outputs->polar is NULL");
    if (out->hits && !aligned16(out->hits)) return fail(ctx, SONAR_ERR_ARG, "hits must be 16-byte aligned");
    if (out->fan && (out->fan_w < 1 || out->fan_h < 1)) return fail(ctx, SONAR_ERR_ARG, "fan size must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    const Tune t = single_tune(ctx, *sensor);
    SensorDev S = make_sensor(*sensor, seed, frame, t, out->fan ? out->fan_w : 0, out->fan ? out->fan_h : 0);
    const int64_t npol = (int64_t)S.nr * S.naz;
    float* noised = out->noised;
    if (!noised) {
        CU(grow(ctx->noised, sizeof(float) * npol, s), "scratch allocation");
        noised = (float*)ctx->noised.p;
    }
    CU(grow(ctx->rowmax, sizeof(uint32_t), s), "scratch allocation");
    sonar_hit* hits = out->hits;
    if (!hits) {
        CU(grow(ctx->hits, sizeof(sonar_hit) * (size_t)S.nb * S.ne, s), "scratch allocation");
        hits = (sonar_hit*)ctx->hits.p;
    }
    CU(grow_trig(ctx, (size_t)(S.nb + S.ne), s), "scratch allocation");
    S.trig = (float4*)ctx->trig.p;
    sonar_status st2 = single_forward(ctx, S, scene_dev(ctx->scenes[scene_id]), params, d_theta, n_mat, hits, noised,
                                      out->binned, (uint32_t*)ctx->rowmax.p, t.block, s);
    if (st2 != SONAR_OK) return st2;
    (void)npol;
    return single_post(ctx, S, params->normalise, noised, (const uint32_t*)ctx->rowmax.p, out->polar, out->fan, s);
}

extern "C" sonar_status sonar_fan_resample(sonar_ctx_t ctx, const sonar_sensor* sensor, const float* d_polar,
                                           int32_t fan_w, int32_t fan_h, float* d_fan, void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    sonar_status st = check_sensor(ctx, sensor);
    if (st) return st;
    if (!d_polar || !d_fan) return fail(ctx, SONAR_ERR_ARG, "NULL polar or fan");
    if (fan_w < 1 || fan_h < 1) return fail(ctx, SONAR_ERR_ARG, "fan size must be >= 1");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    Tune t;
    t.cols = 1;
    const SensorDev S = make_sensor(*sensor, 0, 0, t, fan_w, fan_h);
    FanArgs f{};
    f.one = S;
    f.polar = d_polar;
    f.fan = d_fan;
    CU(launch_fan_tiles(f, tile_squares(S.fan_w, S.fan_h), (cudaStream_t)stream), "fan launch");
    return SONAR_OK;
}

extern "C" sonar_status sonar_render_backward(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                                              const sonar_params* params, const float* d_theta, int32_t n_mat,
                                              uint64_t seed, uint64_t frame, const float* d_grad_polar,
                                              const float* d_noised, const sonar_hit* d_hits, float* d_dtheta,
                                              void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    sonar_status st;
    if ((st = check_scene(ctx, scene_id)) || (st = check_sensor(ctx, sensor)) || (st = check_params(ctx, params)) ||
        (st = check_nmat(ctx, scene_id, n_mat)))
        return st;
    if (!d_theta || !d_grad_polar || !d_noised || !d_dtheta)
        return fail(ctx, SONAR_ERR_ARG, "NULL theta, grad, noised or dtheta");
    if (d_hits && !aligned16(d_hits)) return fail(ctx, SONAR_ERR_ARG, "hits must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    const Tune t = tune_for(ctx, *sensor);
    SensorDev S = make_sensor(*sensor, seed, frame, t, 0, 0);
    const int groups = params->normalise == 1 ? S.nr : 1;
    CU(grow(ctx->rowinfo, sizeof(RowInfo) * groups, s), "scratch allocation");
    const sonar_hit* hits = d_hits;
    if (!hits) {   // recompute the hit records with the ray-cast kernel (bitwise the forward's)
        CU(grow_trig(ctx, (size_t)(S.nb + S.ne), s), "scratch allocation");
        CU(grow(ctx->hits, sizeof(sonar_hit) * (size_t)S.nb * S.ne, s), "scratch allocation");
        S.trig = (float4*)ctx->trig.p;
        S.occ = single_variant(ctx, *sensor, S.tb, S.occ);
        CU(single_trig(ctx, S, s), "trig launch");
        TraceArgs tr{};
        tr.one = S;
        tr.one_scene = scene_dev(ctx->scenes[scene_id]);
        tr.params = *params;
        tr.hits = (sonar_hit*)ctx->hits.p;
        tr.err = ctx->d_err;
        CU(launch_trace(tr, S.trace_blocks, S.occ, s), "trace launch");
        hits = (const sonar_hit*)ctx->hits.p;
    }
    const int nq = n_mat + 2;
    const int64_t rays = (int64_t)S.nb * S.ne;
    const int chunk = adj_chunk(rays, ctx->sm_count, t.block);
    const int n_units = (int)((rays + chunk - 1) / chunk);
    CU(grow(ctx->partials, sizeof(double) * (size_t)n_units * nq, s), "scratch allocation");
    if (params->normalise != 0)
        CU(launch_adj_rows(nullptr, nullptr, S, 1, groups, params->normalise, d_noised, d_grad_polar,
                           (RowInfo*)ctx->rowinfo.p, nullptr, s),
           "adjoint row launch");
    AdjArgs a{};
    a.n_units = n_units;
    a.chunk = chunk;
    a.n_mat = n_mat;
    a.one = S;
    a.one_scene = scene_dev(ctx->scenes[scene_id]);
    a.theta = d_theta;
    a.params = *params;
    a.grad = d_grad_polar;
    a.hits = hits;
    a.rowinfo = (const RowInfo*)ctx->rowinfo.p;
    a.partials = (double*)ctx->partials.p;
    a.err = ctx->d_err;
    const size_t smem = sizeof(double) * (t.block / 32) * n_mat;
    CU(launch_adjoint(a, n_units, t.block, smem, d_dtheta, s), "adjoint launch");
    return SONAR_OK;
}

// ===========================================================================
// batches
// ===========================================================================

struct sonar_batch {
    sonar_ctx* ctx = nullptr;
    std::vector<sonar_batch_item> items;
    std::vector<SensorDev> hs;        // host copy of the descriptors
    std::vector<Unit> units;          // forward work list (column tiles)
    std::vector<AdjUnit> adj_units;   // adjoint work list (ray chunks)
    std::vector<int32_t> fan_prefix;  // fan blocks per sensor, prefix
    std::vector<int32_t> trace_prefix;  // trace blocks per sensor, prefix
    int64_t total_rays = 0;
    int64_t total_rows = 0, total_polar = 0;
    int block = 128;
    int trace_occ = 0;
    int adj_chunk = 0;
    size_t smem1 = 0;
    SensorDev* d_sens = nullptr;
    Unit* d_units = nullptr;
    AdjUnit* d_adj_units = nullptr;
    SceneDev* d_scenes = nullptr;
    int32_t* d_fan_prefix = nullptr;
    int32_t* d_trace_prefix = nullptr;
    int4* d_trace_map = nullptr;      // per trace block: (sensor, tile, scene, 0)
    std::vector<int4> h_trace_map;    // its host copy (an update that moves an item to another scene patches it)
    int2* d_fan_map = nullptr;        // per fan block: (sensor, block)
    int32_t* d_row_map = nullptr;     // per range row: sensor
    // fan coordinate tables: sensors with the same fan geometry share one,
    // filled from the owner's descriptor on every forward replay
    std::vector<int> lut_owner;       // per sensor: owner of its table (-1: none)
    std::vector<uint4*> lut_of;       // per sensor: the table of its owner (nullptr: none)
    uint4* d_fan_lut = nullptr;       // all tables
    uint4** d_luts = nullptr;         // per sensor: its own table when it is an owner
    int2* d_lut_map = nullptr;        // per table block: (owner, block)
    int4* d_group_map = nullptr;      // per grouped fan block: (owner, pixel block, users [m0, m1))
    int32_t* d_members = nullptr;     // users of each table, by owner
    uint32_t* d_fan_stamp = nullptr;  // per table block: the owner's fan_version it was built for
    int lut_blocks = 0, group_blocks = 0;
    int fan_blocks = 0;               // blocks of the per-sensor fan launch
    sonar_hit* d_hits = nullptr;      // hit records when the caller asks for none
    float4* d_trig = nullptr;         // per-sensor exact-ray tables
    uint32_t* d_trig_stamp = nullptr; // per sensor and k_trig block: the version its entries were built for
    int max_angles = 0;
    uint32_t* d_rowmax = nullptr;
    float* d_noised = nullptr;
    RowInfo* d_rowinfo = nullptr;
    double* d_partials = nullptr;
    int32_t* d_counters = nullptr;    // [0] phase-1 work, [1] adjoint work
    int n_mat_cap = 0;
    size_t n_scene_table = 0;         // entries in d_scenes
    // host staging for updates (pinned, double-buffered)
    SensorDev* h_stage[2] = {nullptr, nullptr};
    SceneDev* h_stage_sc[2] = {nullptr, nullptr};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int stage_next = 0;
    // graphs
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;      // the adjoint branch of the combined step graph
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaGraphExec_t fwd = nullptr, bwd = nullptr, step = nullptr;
    // the forward without the two table kernels (exact-ray sin/cos, fan
    // coordinates), replayed while the tables are known to be current: no
    // update or plan since a forward that built them was enqueued (the fan
    // coordinates are built only by a forward that writes fans)
    cudaGraphExec_t fwd_lean = nullptr;
    bool trig_current = false, lut_current = false;
    bool lean_last = false;           // the last forward replay was the lean graph
    cudaEvent_t ev[7] = {};           // phase boundaries recorded inside the graphs
    bool ran_fwd = false, ran_bwd = false;
    std::vector<unsigned char> fwd_key, fwd_lean_key, bwd_key, step_key;
    int graphs = 0;
    int fwd_kernels = 0, fwd_lean_kernels = 0, bwd_kernels = 0, step_kernels = 0;   // kernel nodes of the current graphs
};

namespace {

void batch_free_device(sonar_batch* b) {
    for (void* p : {(void*)b->d_sens, (void*)b->d_units, (void*)b->d_adj_units, (void*)b->d_scenes,
                    (void*)b->d_fan_prefix, (void*)b->d_trace_prefix, (void*)b->d_trace_map,
                    (void*)b->d_fan_map, (void*)b->d_row_map, (void*)b->d_hits, (void*)b->d_trig, (void*)b->d_trig_stamp,
                    (void*)b->d_rowmax,
                    (void*)b->d_noised, (void*)b->d_rowinfo, (void*)b->d_partials, (void*)b->d_counters,
                    (void*)b->d_fan_lut, (void*)b->d_luts, (void*)b->d_lut_map, (void*)b->d_group_map,
                    (void*)b->d_members, (void*)b->d_fan_stamp})
        if (p) cudaFree(p);
    b->d_fan_lut = nullptr;
    b->d_luts = nullptr;
    b->d_lut_map = nullptr;
    b->d_group_map = nullptr;
    b->d_members = nullptr;
    b->d_fan_stamp = nullptr;
    b->lut_blocks = b->group_blocks = b->fan_blocks = 0;
    b->d_trace_prefix = nullptr;
    b->d_trace_map = nullptr;
    b->d_fan_map = nullptr;
    b->d_row_map = nullptr;
    b->d_hits = nullptr;
    b->d_trig = nullptr;
    b->d_trig_stamp = nullptr;
    b->n_mat_cap = 0;
    b->d_sens = nullptr; b->d_units = nullptr; b->d_adj_units = nullptr; b->d_scenes = nullptr;
    b->d_fan_prefix = nullptr;
    b->d_rowmax = nullptr; b->d_noised = nullptr; b->d_rowinfo = nullptr; b->d_partials = nullptr;
    b->d_counters = nullptr;
    if (b->fwd) cudaGraphExecDestroy(b->fwd);
    if (b->fwd_lean) cudaGraphExecDestroy(b->fwd_lean);
    if (b->bwd) cudaGraphExecDestroy(b->bwd);
    if (b->step) cudaGraphExecDestroy(b->step);
    b->fwd = b->fwd_lean = b->bwd = b->step = nullptr;
    b->fwd_key.clear();
    b->fwd_lean_key.clear();
    b->bwd_key.clear();
    b->step_key.clear();
    b->trig_current = b->lut_current = false;
}

// Fan pixels sample the same bins with the same weights exactly when these agree.
bool same_fan_geometry(const SensorDev& x, const SensorDev& y) {
    auto eq = [](float a, float b) { return memcmp(&a, &b, sizeof a) == 0; };
    return x.nr == y.nr && x.naz == y.naz && x.fan_w == y.fan_w && x.fan_h == y.fan_h && eq(x.hfov, y.hfov) &&
           eq(x.rmin, y.rmin) && eq(x.rmax, y.rmax) && eq(x.inv_dr, y.inv_dr) && eq(x.fan_scale, y.fan_scale);
}

std::vector<SceneDev> scene_table(const sonar_ctx* ctx) {
    std::vector<SceneDev> t(ctx->scenes.size());
    for (size_t k = 0; k < t.size(); ++k) t[k] = scene_dev(ctx->scenes[k]);
    return t;
}

sonar_status check_items(sonar_ctx* ctx, const sonar_batch_item* items, int32_t n) {
    if (!items || n < 1) return fail(ctx, SONAR_ERR_ARG, "batch needs at least one item");
    for (int k = 0; k < n; ++k) {
        sonar_status st;
        if ((st = check_scene(ctx, items[k].scene_id)) || (st = check_sensor(ctx, &items[k].sensor))) {
            ctx->last_error = "item " + std::to_string(k) + ": " + ctx->last_error;
            return st;
        }
        if (items[k].fan_w < 0 || items[k].fan_h < 0 || (items[k].fan_w > 0) != (items[k].fan_h > 0))
            return fail(ctx, SONAR_ERR_ARG, "item " + std::to_string(k) + ": bad fan size");
        if (items[k].polar_offset < 0 || items[k].hits_offset < 0 || items[k].fan_offset < 0)
            return fail(ctx, SONAR_ERR_ARG, "item " + std::to_string(k) + ": negative offset");
    }
    return SONAR_OK;
}

// (Re)builds descriptors, work units and device buffers from b->items.
sonar_status batch_plan(sonar_batch* b) {
    sonar_ctx* ctx = b->ctx;
    batch_free_device(b);
    const int n = (int)b->items.size();
    b->hs.assign(n, SensorDev{});
    b->units.clear();
    b->adj_units.clear();
    b->fan_prefix.assign(n + 1, 0);
    b->trace_prefix.assign(n + 1, 0);
    b->smem1 = 0;
    int64_t rows = 0, polar_end = 0;
    std::map<int, int64_t> block_votes;
    for (int k = 0; k < n; ++k) {
        const sonar_batch_item& it = b->items[k];
        const Tune t = tune_for(ctx, it.sensor);
        SensorDev S = make_sensor(it.sensor, it.seed, it.frame, t, it.fan_w, it.fan_h);
        S.scene = it.scene_id;
        S.polar_off = it.polar_offset;
        S.hits_off = it.hits_offset;
        S.fan_off = it.fan_offset;
        S.rowmax_off = rows;
        rows += S.nr;    // room for mode 1; mode 2 uses the first slot of each sensor
        polar_end = std::max<int64_t>(polar_end, it.polar_offset + (int64_t)S.nr * S.naz);
        b->hs[k] = S;
        b->fan_prefix[k + 1] =
            b->fan_prefix[k] + (S.fan_w > 0 ? tile_squares(S.fan_w, S.fan_h) : 0);
        b->trace_prefix[k + 1] = b->trace_prefix[k] + S.trace_blocks;
        block_votes[t.block] += (int64_t)S.nb * S.ne;
        for (int tile = 0; tile < S.n_tiles; ++tile) {
            Unit u;
            u.sensor = k;
            u.scene = S.scene;
            u.c0 = tile * S.cols;
            u.c1 = std::min(u.c0 + S.cols, S.naz);
            const int64_t i0 = first_beam_of_col(u.c0, S.nb, S.naz), i1 = first_beam_of_col(u.c1, S.nb, S.naz);
            u.rays = (int32_t)((i1 - i0) * S.ne);
            b->units.push_back(u);
        }
        b->smem1 = std::max(b->smem1, bin_smem(S));
    }
    // largest units first: the persistent blocks then finish close together
    std::stable_sort(b->units.begin(), b->units.end(), [&](const Unit& x, const Unit& y) {
        return (int64_t)x.rays * 4 + b->hs[x.sensor].nr * (x.c1 - x.c0) / 64 >
               (int64_t)y.rays * 4 + b->hs[y.sensor].nr * (y.c1 - y.c0) / 64;
    });
    b->block = 128;
    int64_t best = -1;
    for (auto& kv : block_votes)
        if (kv.second > best) { best = kv.second; b->block = kv.first; }
    // the trace launch takes the variant of the sensor shape with most rays; an
    // untuned shape walks the tree the launch size calls for, and the 8-wide tree
    // only when every scene of the batch has one
    int64_t most = -1;
    int kmost = 0;
    for (int k = 0; k < n; ++k) {
        const SensorDev& S = b->hs[k];
        if ((int64_t)S.nb * S.ne > most) { most = (int64_t)S.nb * S.ne; b->trace_occ = S.occ; kmost = k; }
    }
    if (n > 0) {
        const sonar_sensor& ms = b->items[kmost].sensor;
        if (!ctx->tune.count(ShapeKey{ms.n_beams, ms.n_elev, ms.n_range_bins, ms.n_az_bins}))
            b->trace_occ = (b->trace_occ & ~kTraceWide) | wide_for_launch(ctx, b->trace_prefix[n]);
        for (const sonar_batch_item& it : b->items)
            if (!ctx->scenes[it.scene_id].nodes8) b->trace_occ &= ~kTraceWide;
    }
    b->total_rows = rows;
    b->total_polar = polar_end;
    int64_t all_rays = 0;
    for (const SensorDev& S : b->hs) all_rays += (int64_t)S.nb * S.ne;
    b->total_rays = all_rays;
    b->adj_chunk = adj_chunk(all_rays, ctx->sm_count, b->block);
    for (int k = 0; k < n; ++k) {
        const int64_t r = (int64_t)b->hs[k].nb * b->hs[k].ne;
        for (int64_t r0 = 0; r0 < r; r0 += b->adj_chunk)
            b->adj_units.push_back(AdjUnit{k, (int32_t)r0, (int32_t)std::min<int64_t>(r, r0 + b->adj_chunk),
                                           b->hs[k].scene});
    }
    const size_t nu = b->units.size(), na = b->adj_units.size();
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max(bytes, (size_t)16));
    };
    alloc((void**)&b->d_sens, sizeof(SensorDev) * n);
    alloc((void**)&b->d_units, sizeof(Unit) * nu);
    alloc((void**)&b->d_scenes, sizeof(SceneDev) * std::max<size_t>(1, ctx->scenes.size()));
    b->n_scene_table = ctx->scenes.size();
    alloc((void**)&b->d_adj_units, sizeof(AdjUnit) * na);
    alloc((void**)&b->d_fan_prefix, sizeof(int32_t) * (n + 1));
    alloc((void**)&b->d_trace_prefix, sizeof(int32_t) * (n + 1));
    // fan coordinate tables for geometries that more than one sensor shares
    b->lut_owner.assign(n, -1);
    b->lut_of.assign(n, nullptr);
    std::vector<int> owners;
    std::vector<int> members(n, 0);
    for (int k = 0; k < n; ++k) {
        if (b->hs[k].fan_w <= 0) continue;
        for (int o : owners)
            if (same_fan_geometry(b->hs[k], b->hs[o])) { b->lut_owner[k] = o; ++members[o]; break; }
        if (b->lut_owner[k] < 0) { owners.push_back(k); b->lut_owner[k] = k; members[k] = 1; }
    }
    int64_t lut_px = 0;
    std::vector<int64_t> lut_at(n, -1), stamp_at(n, -1);
    std::vector<int2> lmap;
    for (int o : owners) {
        if (members[o] < 2) continue;
        const int64_t px = (int64_t)b->hs[o].fan_w * b->hs[o].fan_h;
        lut_at[o] = lut_px;
        lut_px += px;
        stamp_at[o] = (int64_t)lmap.size();
        for (int64_t t = 0; t < (px + kFanTile - 1) / kFanTile; ++t) lmap.push_back(make_int2(o, (int)t));
    }
    for (int k = 0; k < n; ++k)
        if (b->lut_owner[k] >= 0 && lut_at[b->lut_owner[k]] < 0) b->lut_owner[k] = -1;
    b->lut_blocks = (int)lmap.size();
    // the fan of a table's users: blocks of (owner, pixel block, run of up to
    // kFanGroup users), so that a table entry serves several frames
    std::vector<int4> gmap;
    std::vector<int32_t> mem;
    for (int o : owners) {
        if (lut_at[o] < 0) continue;
        const int32_t m0 = (int32_t)mem.size();
        for (int k = 0; k < n; ++k)
            if (b->lut_owner[k] == o) mem.push_back(k);
        const int32_t m1 = (int32_t)mem.size();
        for (int32_t a0 = m0; a0 < m1; a0 += kFanGroup)
            for (int t = 0; t < fan_squares(b->hs[o].fan_w, b->hs[o].fan_h); ++t)
                gmap.push_back(make_int4(o, t, a0, std::min(a0 + kFanGroup, m1)));
    }
    b->group_blocks = (int)gmap.size();
    if (lut_px > 0) {
        alloc((void**)&b->d_fan_lut, sizeof(uint4) * lut_px);
        alloc((void**)&b->d_luts, sizeof(uint4*) * n);
        alloc((void**)&b->d_lut_map, sizeof(int2) * lmap.size());
        alloc((void**)&b->d_group_map, sizeof(int4) * gmap.size());
        alloc((void**)&b->d_members, sizeof(int32_t) * mem.size());
        alloc((void**)&b->d_fan_stamp, sizeof(uint32_t) * lmap.size());
        if (e == cudaSuccess) e = cudaMemset(b->d_fan_stamp, 0, sizeof(uint32_t) * lmap.size());
        if (e == cudaSuccess) {
            std::vector<uint4*> own(n, nullptr);
            for (int k = 0; k < n; ++k) {
                const int o = b->lut_owner[k];
                if (o < 0) continue;
                b->lut_of[k] = b->d_fan_lut + lut_at[o];
                b->hs[k].fan_lut = b->lut_of[k];
                if (o == k) {
                    own[k] = b->lut_of[k];
                    b->hs[k].fan_stamp = b->d_fan_stamp + stamp_at[o];   // stamps 0: every block builds once
                    b->hs[k].fan_version = 1;
                }
            }
            e = cudaMemcpy(b->d_luts, own.data(), sizeof(uint4*) * n, cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(b->d_lut_map, lmap.data(), sizeof(int2) * lmap.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(b->d_group_map, gmap.data(), sizeof(int4) * gmap.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(b->d_members, mem.data(), sizeof(int32_t) * mem.size(), cudaMemcpyHostToDevice);
        }
    }
    std::vector<int4> tmap;
    std::vector<int2> fmap;
    std::vector<int32_t> rmap;
    // Ray-cast blocks in eight bands of decreasing upward component (world z) of
    // their tile's central ray, sensor by sensor inside a band.  Over a seabed
    // the rays closest to the horizon run farthest, so the longest blocks start
    // first and the launch's tail is short (longest-processing-time-first); the
    // bands keep a sensor's neighbouring tiles together, which share nodes in L2.
    // Results do not depend on the order.
    {
        std::vector<std::pair<float, int64_t>> order;
        for (int k = 0; k < n; ++k) {
            const SensorDev& S = b->hs[k];
            const int tb = S.tb, te = 32 / S.tb, tiles_b = (S.nb + tb - 1) / tb;
            for (int t = 0; t < S.trace_blocks; ++t) {
                const int ty = t / tiles_b, tx = t - ty * tiles_b;
                const double i = std::min(tx * tb + 0.5 * tb, (double)S.nb);
                const double j = std::min(ty * te + 0.5 * te, (double)S.ne);
                const double phi = i * S.hfov / S.nb - 0.5 * S.hfov, th = j * S.vfov / S.ne - 0.5 * S.vfov;
                const double up = S.rot[6] * std::sin(phi) * std::cos(th) + S.rot[7] * std::cos(phi) * std::cos(th) +
                                  S.rot[8] * std::sin(th);
                order.push_back({(float)-up, ((int64_t)k << 32) | (uint32_t)t});
            }
        }
        if (!order.empty()) {
            constexpr int kBands = 8;
            float lo = order[0].first, hi = order[0].first;
            for (const auto& q : order) { lo = std::min(lo, q.first); hi = std::max(hi, q.first); }
            const float width = (hi - lo) / kBands;
            for (auto& q : order)
                q.first = width > 0.0f ? std::min((float)(kBands - 1), std::floor((q.first - lo) / width)) : 0.0f;
        }
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<float, int64_t>& x, const std::pair<float, int64_t>& y) {
                             return x.first < y.first;
                         });
        for (const auto& q : order) {
            const int k = (int)(q.second >> 32);
            tmap.push_back(make_int4(k, (int)(q.second & 0xFFFFFFFF), b->hs[k].scene, 0));
        }
    }
    for (int k = 0; k < n; ++k) {
        if (b->lut_owner[k] < 0)   // sensors with a shared table are resampled by the grouped launch
            for (int t = 0; t < b->fan_prefix[k + 1] - b->fan_prefix[k]; ++t) fmap.push_back(make_int2(k, t));
        for (int r = 0; r < b->hs[k].nr; ++r) rmap.push_back(k);
    }
    alloc((void**)&b->d_trace_map, sizeof(int4) * tmap.size());
    alloc((void**)&b->d_fan_map, sizeof(int2) * std::max<size_t>(1, fmap.size()));
    b->fan_blocks = (int)fmap.size();
    alloc((void**)&b->d_row_map, sizeof(int32_t) * rmap.size());
    int64_t angles = 0;
    b->max_angles = 0;
    for (const SensorDev& S : b->hs) {
        angles += S.nb + S.ne;
        b->max_angles = std::max(b->max_angles, S.nb + S.ne);
    }
    alloc((void**)&b->d_trig, sizeof(float4) * angles);
    // per sensor, one stamp per k_trig block (grid x = ceil(max_angles / 128)):
    // stamps 0 and versions 1, so every block builds its entries once
    const int trig_gx = (b->max_angles + 127) / 128;
    alloc((void**)&b->d_trig_stamp, sizeof(uint32_t) * std::max<int64_t>(1, (int64_t)n * trig_gx));
    if (e == cudaSuccess) e = cudaMemset(b->d_trig_stamp, 0, sizeof(uint32_t) * std::max<int64_t>(1, (int64_t)n * trig_gx));
    if (e == cudaSuccess) {
        int64_t off = 0;
        for (int k = 0; k < n; ++k) {
            SensorDev& S = b->hs[k];
            S.trig = b->d_trig + off;
            off += S.nb + S.ne;
            S.trig_stamp = b->d_trig_stamp + (int64_t)k * trig_gx;
            S.trig_version = 1;
        }
    }
    alloc((void**)&b->d_rowmax, sizeof(uint32_t) * rows);
    alloc((void**)&b->d_rowinfo, sizeof(RowInfo) * rows);
    alloc((void**)&b->d_counters, sizeof(int32_t) * 4);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch allocation");
    const std::vector<SceneDev> table = scene_table(ctx);
    e = cudaMemcpy(b->d_sens, b->hs.data(), sizeof(SensorDev) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_units, b->units.data(), sizeof(Unit) * nu, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !table.empty())
        e = cudaMemcpy(b->d_scenes, table.data(), sizeof(SceneDev) * table.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_adj_units, b->adj_units.data(), sizeof(AdjUnit) * na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_fan_prefix, b->fan_prefix.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_trace_prefix, b->trace_prefix.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_trace_map, tmap.data(), sizeof(int4) * tmap.size(), cudaMemcpyHostToDevice);
    b->h_trace_map = std::move(tmap);
    if (e == cudaSuccess && !fmap.empty())
        e = cudaMemcpy(b->d_fan_map, fmap.data(), sizeof(int2) * fmap.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_row_map, rmap.data(), sizeof(int32_t) * rmap.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    return SONAR_OK;
}

// Scratch for outputs the caller does not want (noised image, hit records),
// allocated before any capture: an allocation inside stream capture fails.
cudaError_t batch_scratch(sonar_batch* b, const sonar_batch_outputs* out) {
    cudaError_t e = cudaSuccess;
    if (!out->noised && !b->d_noised)
        e = cudaMalloc(&b->d_noised, sizeof(float) * std::max<int64_t>(1, b->total_polar));
    if (e == cudaSuccess && !out->hits && !b->d_hits)
        e = cudaMalloc(&b->d_hits, sizeof(sonar_hit) * std::max<int64_t>(1, b->total_rays));
    return e;
}

int persistent_grid(const sonar_batch* b, int det) {
    const int per_sm = bin_blocks_per_sm(det, b->block, b->smem1);
    const int64_t g = std::min<int64_t>((int64_t)b->units.size(), (int64_t)b->ctx->sm_count * per_sm);
    return (int)std::max<int64_t>(1, g);
}

// Kernel nodes of a captured graph (-1 if the graph cannot be inspected).
int kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n > 0 && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int k = 0;
    for (cudaGraphNode_t v : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(v, &t) != cudaSuccess) return -1;
        k += t == cudaGraphNodeTypeKernel;
    }
    return k;
}

template <class T>
void append_bytes(std::vector<unsigned char>& v, const T& x) {
    const unsigned char* p = (const unsigned char*)&x;
    v.insert(v.end(), p, p + sizeof(T));
}

// The forward's launches: part 1 up to binning (trig tables, ray cast, binning
// and noise), part 2 the normalisation and fan, part 0 both.
sonar_status batch_forward_launches(sonar_batch* b, const sonar_params* p, const float* d_theta, int32_t n_mat,
                                    const sonar_batch_outputs* out, cudaStream_t s, bool events = false,
                                    int part = 0, bool tables = true) {
    sonar_ctx* ctx = b->ctx;
    const int det = p->accumulate == 0;
    if (part != 2) {
        if (p->normalise == 2)
            CU(cudaMemsetAsync(b->d_rowmax, 0, sizeof(uint32_t) * b->total_rows, s), "cudaMemsetAsync");
        sonar_hit* hits = out->hits ? out->hits : b->d_hits;   // scratch allocated by the caller, outside capture
        if (events) CU(cudaEventRecordWithFlags(b->ev[0], s, cudaEventRecordExternal), "cudaEventRecord");
        if (tables)
            CU(launch_trig(b->d_sens, SensorDev{}, (int)b->items.size(), b->max_angles, s), "batch trig launch");
        TraceArgs t{};
        t.sensors = b->d_sens;
        t.scenes = b->d_scenes;
        t.block_map = b->d_trace_map;
        t.n_sensors = (int32_t)b->items.size();
        t.params = *p;
        t.hits = hits;
        t.err = ctx->d_err;
        t.zero_word = b->d_counters;   // the binning's work counter, cleared for the launch after
        CU(launch_trace(t, b->trace_prefix.back(), b->trace_occ, s), "batch trace launch");
        if (events) CU(cudaEventRecordWithFlags(b->ev[6], s, cudaEventRecordExternal), "cudaEventRecord");
        BinArgs a{};
        a.sensors = b->d_sens;
        a.units = b->d_units;
        a.scenes = b->d_scenes;
        a.work_counter = b->d_counters;
        a.n_units = (int32_t)b->units.size();
        a.n_mat = n_mat;
        a.theta = d_theta;
        a.params = *p;
        a.noised = out->noised ? out->noised : b->d_noised;
        a.binned = out->binned;
        a.hits = hits;
        a.rowmax = b->d_rowmax;
        a.err = ctx->d_err;
        CU(launch_bin(a, det, persistent_grid(b, det), b->block, b->smem1, s), "batch binning launch");
        if (events) CU(cudaEventRecordWithFlags(b->ev[1], s, cudaEventRecordExternal), "cudaEventRecord");
    }
    if (part == 1) return SONAR_OK;
    NormArgs c{};
    c.sensors = b->d_sens;
    c.row_map = b->d_row_map;
    c.n_sensors = (int32_t)b->items.size();
    c.total_rows = b->total_rows;
    c.noised = out->noised ? out->noised : b->d_noised;
    c.gmax = b->d_rowmax;
    c.normalise = p->normalise;
    c.polar = out->polar;
    CU(launch_norm(c, s), "batch normalisation launch");
    if (out->fan) {
        FanArgs f{};
        f.sensors = b->d_sens;
        f.block_map = b->d_fan_map;
        f.n_sensors = (int32_t)b->items.size();
        f.polar = out->polar;
        f.fan = out->fan;
        if (b->lut_blocks > 0) {
            if (tables) {
                FanLutArgs l{b->d_sens, b->d_lut_map, b->d_luts};
                CU(launch_fan_lut(l, b->lut_blocks, s), "batch fan table launch");
            }
            FanGroupArgs g{b->d_sens, b->d_group_map, b->d_members, out->polar, out->fan};
            CU(launch_fan_group(g, b->group_blocks, s), "batch grouped fan launch");
        }
        CU(launch_fan_tiles(f, b->fan_blocks, s), "batch fan launch");
    }
    if (events) CU(cudaEventRecordWithFlags(b->ev[2], s, cudaEventRecordExternal), "cudaEventRecord");
    return SONAR_OK;
}

}  // namespace

extern "C" sonar_status sonar_batch_create(sonar_ctx_t ctx, const sonar_batch_item* items, int32_t n,
                                           sonar_batch_t* out) {
    if (!ctx || !out) return fail(ctx, SONAR_ERR_ARG, "NULL argument");
    *out = nullptr;
    sonar_status st = check_items(ctx, items, n);
    if (st) return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    sonar_batch* b = new sonar_batch();
    b->ctx = ctx;
    b->items.assign(items, items + n);
    st = batch_plan(b);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && st == SONAR_OK; ++k) {
        if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_stage[k], sizeof(SensorDev) * n);
        if (e == cudaSuccess)
            e = cudaMallocHost((void**)&b->h_stage_sc[k], sizeof(SceneDev) * std::max<size_t>(1, 64));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->stage_ev[k], cudaEventDisableTiming);
    }
    if (st == SONAR_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (st == SONAR_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (st == SONAR_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (st == SONAR_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming);
    for (int k = 0; k < 7 && st == SONAR_OK && e == cudaSuccess; ++k) e = cudaEventCreate(&b->ev[k]);
    if (st == SONAR_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "batch staging");
    if (st != SONAR_OK) {
        sonar_batch_destroy(b);
        return st;
    }
    *out = b;
    return SONAR_OK;
}

extern "C" sonar_status sonar_batch_update(sonar_batch_t b, const sonar_batch_item* items, int32_t n, void* stream) {
    if (!b) return SONAR_ERR_ARG;
    b->trig_current = b->lut_current = false;   // the next forward replays the table kernels (they skip current entries)
    sonar_ctx* ctx = b->ctx;
    sonar_status st = check_items(ctx, items, n);
    if (st) return st;
    if (n != (int32_t)b->items.size()) return fail(ctx, SONAR_ERR_ARG, "item count differs from the plan");
    for (int k = 0; k < n; ++k) {
        const sonar_batch_item& x = items[k];
        const sonar_batch_item& y = b->items[k];
        if (x.sensor.n_beams != y.sensor.n_beams || x.sensor.n_elev != y.sensor.n_elev ||
            x.sensor.n_range_bins != y.sensor.n_range_bins || x.sensor.n_az_bins != y.sensor.n_az_bins ||
            x.fan_w != y.fan_w || x.fan_h != y.fan_h || x.polar_offset != y.polar_offset ||
            x.hits_offset != y.hits_offset || x.fan_offset != y.fan_offset)
            return fail(ctx, SONAR_ERR_ARG, "item " + std::to_string(k) + ": shape or offsets differ from the plan");
    }
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    bool new_scene = false;
    for (int k = 0; k < n; ++k) new_scene |= (size_t)items[k].scene_id >= b->n_scene_table;
    if (new_scene) {
        // a scene uploaded after planning: rebuild the scene table (synchronous)
        CU(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronisation");
        const std::vector<SceneDev> table = scene_table(ctx);
        SceneDev* d = nullptr;
        CU(cudaMalloc(&d, sizeof(SceneDev) * table.size()), "scene table");
        CU(cudaMemcpy(d, table.data(), sizeof(SceneDev) * table.size(), cudaMemcpyHostToDevice), "scene table");
        cudaFree(b->d_scenes);
        b->d_scenes = d;
        b->n_scene_table = table.size();
        if (b->fwd) cudaGraphExecDestroy(b->fwd);
        if (b->fwd_lean) cudaGraphExecDestroy(b->fwd_lean);
        if (b->bwd) cudaGraphExecDestroy(b->bwd);
        b->fwd = b->fwd_lean = b->bwd = nullptr;
    }
    const int slot = b->stage_next;
    b->stage_next ^= 1;
    CU(cudaEventSynchronize(b->stage_ev[slot]), "staging wait");
    bool scene_moved = false;
    for (int k = 0; k < n; ++k) {
        SensorDev S = b->hs[k];
        scene_moved |= S.scene != items[k].scene_id;
        const sonar_batch_item& it = items[k];
        const SensorDev fresh = make_sensor(it.sensor, it.seed, it.frame, Tune{S.cols, S.tb, b->block, S.occ},
                                            it.fan_w, it.fan_h);
        memcpy(S.pos, fresh.pos, sizeof S.pos);
        memcpy(S.rot, fresh.rot, sizeof S.rot);
        S.hfov = fresh.hfov; S.vfov = fresh.vfov; S.rmin = fresh.rmin; S.rmax = fresh.rmax;
        S.inv_dr = fresh.inv_dr; S.fan_scale = fresh.fan_scale;
        S.seed_lo = fresh.seed_lo; S.seed_hi = fresh.seed_hi; S.frame_lo = fresh.frame_lo; S.frame_hi = fresh.frame_hi;
        S.scene = it.scene_id;
        // an owner's table is rebuilt (inside the graph) once its fan geometry changes
        if (S.fan_stamp && !same_fan_geometry(S, b->hs[k]) && ++S.fan_version == 0) S.fan_version = 1;   // 0: never built
        // and the exact-ray tables once a field of view changes
        if (S.trig_stamp && (S.hfov != b->hs[k].hfov || S.vfov != b->hs[k].vfov) && ++S.trig_version == 0)
            S.trig_version = 1;
        b->hs[k] = S;
        b->items[k] = it;
    }
    for (int k = 0; k < n; ++k) {
        // a sensor keeps its owner's coordinate table only while their fan geometry agrees
        const int o = b->lut_owner.empty() ? -1 : b->lut_owner[k];
        b->hs[k].fan_lut = (o >= 0 && same_fan_geometry(b->hs[k], b->hs[o])) ? b->lut_of[k] : nullptr;
        b->h_stage[slot][k] = b->hs[k];
    }
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(b->d_sens, b->h_stage[slot], sizeof(SensorDev) * n, cudaMemcpyHostToDevice, s),
       "descriptor upload");
    if (scene_moved) {   // the ray-cast map and the work units carry their scene: patch them (rare, pageable copies)
        for (int4& m : b->h_trace_map) m.z = b->hs[m.x].scene;
        for (Unit& x : b->units) x.scene = b->hs[x.sensor].scene;
        for (AdjUnit& x : b->adj_units) x.scene = b->hs[x.sensor].scene;
        CU(cudaMemcpyAsync(b->d_trace_map, b->h_trace_map.data(), sizeof(int4) * b->h_trace_map.size(),
                           cudaMemcpyHostToDevice, s),
           "trace map upload");
        CU(cudaMemcpyAsync(b->d_units, b->units.data(), sizeof(Unit) * b->units.size(), cudaMemcpyHostToDevice, s),
           "unit upload");
        CU(cudaMemcpyAsync(b->d_adj_units, b->adj_units.data(), sizeof(AdjUnit) * b->adj_units.size(),
                           cudaMemcpyHostToDevice, s),
           "unit upload");
    }
    CU(cudaEventRecord(b->stage_ev[slot], s), "cudaEventRecord");
    return SONAR_OK;
}

extern "C" sonar_status sonar_render_batch(sonar_batch_t b, const sonar_params* p, const float* d_theta,
                                           int32_t n_mat, const sonar_batch_outputs* out, void* stream) {
    if (!b) return SONAR_ERR_ARG;
    sonar_ctx* ctx = b->ctx;
    sonar_status st = check_params(ctx, p);
    if (st) return st;
    if (!d_theta || !out || !out->polar) return fail(ctx, SONAR_ERR_ARG, "NULL theta or outputs");
    if (out->hits && !aligned16(out->hits)) return fail(ctx, SONAR_ERR_ARG, "hits must be 16-byte aligned");
    for (const sonar_batch_item& it : b->items)
        if ((st = check_scene(ctx, it.scene_id)) || (st = check_nmat(ctx, it.scene_id, n_mat))) return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    CU(batch_scratch(b, out), "batch scratch");
    std::vector<unsigned char> key;
    append_bytes(key, *p);
    append_bytes(key, d_theta);
    append_bytes(key, n_mat);
    append_bytes(key, *out);
    // the full forward while a table it reads may be stale, else the lean one
    const bool lean = b->trig_current && (b->lut_current || !out->fan || b->lut_blocks == 0);
    cudaGraphExec_t& exec = lean ? b->fwd_lean : b->fwd;
    std::vector<unsigned char>& exec_key = lean ? b->fwd_lean_key : b->fwd_key;
    if (!exec || key != exec_key) {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "graph capture");
        st = batch_forward_launches(b, p, d_theta, n_mat, out, b->cap, true, 0, !lean);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (st != SONAR_OK) { if (g) cudaGraphDestroy(g); return st; }
        CU(e, "graph capture");
        (lean ? b->fwd_lean_kernels : b->fwd_kernels) = kernel_nodes(g);
        const cudaError_t e2 = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        CU(e2, "graph instantiation");
        exec_key = key;
        ++b->graphs;
    }
    CU(cudaGraphLaunch(exec, s), "graph launch");
    b->trig_current = true;   // built by this replay, in stream order, if they were stale
    if (out->fan) b->lut_current = true;
    b->lean_last = lean;
    b->ran_fwd = true;
    return SONAR_OK;
}

namespace {

sonar_status batch_backward_launches(sonar_batch* b, const sonar_params* p, const float* d_theta, int32_t n_mat,
                                     const float* grad, const float* noised, const sonar_hit* hits, float* dtheta,
                                     cudaStream_t s, bool events = false) {
    sonar_ctx* ctx = b->ctx;
    // the gather's work counter is cleared by a kernel before it (the ray cast
    // of recomputed records, the row terms), else by a memset
    if (hits && p->normalise == 0)
        CU(cudaMemsetAsync(b->d_counters + 1, 0, sizeof(int32_t), s), "cudaMemsetAsync");
    if (events) CU(cudaEventRecordWithFlags(b->ev[3], s, cudaEventRecordExternal), "cudaEventRecord");
    if (!hits) {   // recompute the hit records with the ray-cast kernel into the batch scratch
        CU(launch_trig(b->d_sens, SensorDev{}, (int)b->items.size(), b->max_angles, s), "batch trig launch");
        TraceArgs tr{};
        tr.sensors = b->d_sens;
        tr.scenes = b->d_scenes;
        tr.block_map = b->d_trace_map;
        tr.n_sensors = (int32_t)b->items.size();
        tr.params = *p;
        tr.hits = b->d_hits;
        tr.err = ctx->d_err;
        tr.zero_word = b->d_counters + 1;
        CU(launch_trace(tr, b->trace_prefix.back(), b->trace_occ, s), "batch trace launch");
        hits = b->d_hits;
    }
    if (p->normalise != 0)
        CU(launch_adj_rows(b->d_sens, b->d_row_map, SensorDev{}, (int)b->items.size(),
                           p->normalise == 1 ? b->total_rows : (int64_t)b->items.size(), p->normalise, noised,
                           grad, b->d_rowinfo, b->d_counters + 1, s),
           "batch adjoint rows");
    if (events) CU(cudaEventRecordWithFlags(b->ev[4], s, cudaEventRecordExternal), "cudaEventRecord");
    AdjArgs a{};
    a.sensors = b->d_sens;
    a.units = b->d_adj_units;
    a.scenes = b->d_scenes;
    a.work_counter = b->d_counters + 1;
    a.n_units = (int32_t)b->adj_units.size();
    a.chunk = b->adj_chunk;
    a.n_mat = n_mat;
    a.theta = d_theta;
    a.params = *p;
    a.grad = grad;
    a.hits = hits;
    a.rowinfo = b->d_rowinfo;
    a.partials = b->d_partials;
    a.err = ctx->d_err;
    const size_t smem = sizeof(double) * (b->block / 32) * n_mat;
    const int per_sm = adjoint_blocks_per_sm(b->block, smem);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->adj_units.size(),
                                                                    (int64_t)ctx->sm_count * per_sm));
    CU(launch_adjoint(a, grid, b->block, smem, dtheta, s), "batch adjoint launch");
    if (events) CU(cudaEventRecordWithFlags(b->ev[5], s, cudaEventRecordExternal), "cudaEventRecord");
    return SONAR_OK;
}

}  // namespace

extern "C" sonar_status sonar_render_batch_backward(sonar_batch_t b, const sonar_params* p, const float* d_theta,
                                                    int32_t n_mat, const float* d_grad, const float* d_noised,
                                                    const sonar_hit* d_hits, float* d_dtheta, void* stream) {
    if (!b) return SONAR_ERR_ARG;
    sonar_ctx* ctx = b->ctx;
    sonar_status st = check_params(ctx, p);
    if (st) return st;
    if (!d_theta || !d_grad || !d_noised || !d_dtheta) return fail(ctx, SONAR_ERR_ARG, "NULL argument");
    if (d_hits && !aligned16(d_hits)) return fail(ctx, SONAR_ERR_ARG, "hits must be 16-byte aligned");
    for (const sonar_batch_item& it : b->items)
        if ((st = check_scene(ctx, it.scene_id)) || (st = check_nmat(ctx, it.scene_id, n_mat))) return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!d_hits && !b->d_hits)   // recomputed records need the scratch; allocate outside capture
        CU(cudaMalloc(&b->d_hits, sizeof(sonar_hit) * std::max<int64_t>(1, b->total_rays)), "batch scratch");
    if (n_mat > b->n_mat_cap) {
        if (b->d_partials) cudaFree(b->d_partials);
        b->d_partials = nullptr;
        CU(cudaMalloc(&b->d_partials, sizeof(double) * b->adj_units.size() * (n_mat + 2)), "batch scratch");
        b->n_mat_cap = n_mat;
        if (b->bwd) cudaGraphExecDestroy(b->bwd);
        b->bwd = nullptr;
    }
    std::vector<unsigned char> key;
    append_bytes(key, *p);
    append_bytes(key, d_theta);
    append_bytes(key, n_mat);
    append_bytes(key, d_grad);
    append_bytes(key, d_noised);
    append_bytes(key, d_hits);
    append_bytes(key, d_dtheta);
    if (!b->bwd || key != b->bwd_key) {
        if (b->bwd) cudaGraphExecDestroy(b->bwd);
        b->bwd = nullptr;
        CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "graph capture");
        st = batch_backward_launches(b, p, d_theta, n_mat, d_grad, d_noised, d_hits, d_dtheta, b->cap, true);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (st != SONAR_OK) { if (g) cudaGraphDestroy(g); return st; }
        CU(e, "graph capture");
        b->bwd_kernels = kernel_nodes(g);
        const cudaError_t e2 = cudaGraphInstantiate(&b->bwd, g, 0);
        cudaGraphDestroy(g);
        CU(e2, "graph instantiation");
        b->bwd_key = key;
        ++b->graphs;
    }
    CU(cudaGraphLaunch(b->bwd, (cudaStream_t)stream), "graph launch");
    b->ran_bwd = true;
    return SONAR_OK;
}

extern "C" sonar_status sonar_render_batch_step(sonar_batch_t b, const sonar_params* p, const float* d_theta,
                                                int32_t n_mat, const sonar_batch_outputs* out, const float* d_grad,
                                                float* d_dtheta, void* stream) {
    if (!b) return SONAR_ERR_ARG;
    sonar_ctx* ctx = b->ctx;
    sonar_status st = check_params(ctx, p);
    if (st) return st;
    if (!d_theta || !out || !out->polar || !d_grad || !d_dtheta)
        return fail(ctx, SONAR_ERR_ARG, "NULL theta, outputs, grad or dtheta");
    if (out->hits && !aligned16(out->hits)) return fail(ctx, SONAR_ERR_ARG, "hits must be 16-byte aligned");
    for (const sonar_batch_item& it : b->items)
        if ((st = check_scene(ctx, it.scene_id)) || (st = check_nmat(ctx, it.scene_id, n_mat))) return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    CU(batch_scratch(b, out), "batch scratch");
    if (!out->hits && !b->d_hits)   // the adjoint reads the records the forward writes
        CU(cudaMalloc(&b->d_hits, sizeof(sonar_hit) * std::max<int64_t>(1, b->total_rays)), "batch scratch");
    if (n_mat > b->n_mat_cap) {
        if (b->d_partials) cudaFree(b->d_partials);
        b->d_partials = nullptr;
        CU(cudaMalloc(&b->d_partials, sizeof(double) * b->adj_units.size() * (n_mat + 2)), "batch scratch");
        b->n_mat_cap = n_mat;
        if (b->bwd) cudaGraphExecDestroy(b->bwd);
        if (b->step) cudaGraphExecDestroy(b->step);
        b->bwd = b->step = nullptr;
    }
    std::vector<unsigned char> key;
    append_bytes(key, *p);
    append_bytes(key, d_theta);
    append_bytes(key, n_mat);
    append_bytes(key, *out);
    append_bytes(key, d_grad);
    append_bytes(key, d_dtheta);
    if (!b->step || key != b->step_key) {
        if (b->step) cudaGraphExecDestroy(b->step);
        b->step = nullptr;
        const float* noised = out->noised ? out->noised : b->d_noised;
        const sonar_hit* hits = out->hits ? out->hits : b->d_hits;
        // one graph, two branches after binning: the adjoint (which reads I~ and
        // the hit records only) beside the normalisation and the fan
        CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "graph capture");
        st = batch_forward_launches(b, p, d_theta, n_mat, out, b->cap, true, 1);
        cudaError_t e = cudaSuccess;
        bool forked = false;
        if (st == SONAR_OK) {
            e = cudaEventRecord(b->fork_ev, b->cap);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork_ev, 0);
            forked = e == cudaSuccess;
        }
        if (st == SONAR_OK && forked)
            st = batch_backward_launches(b, p, d_theta, n_mat, d_grad, noised, hits, d_dtheta, b->side, true);
        if (st == SONAR_OK && forked) st = batch_forward_launches(b, p, d_theta, n_mat, out, b->cap, true, 2);
        if (forked) {   // join the branch whatever happened, so that the capture can end
            const cudaError_t e1 = cudaEventRecord(b->join_ev, b->side);
            const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(b->cap, b->join_ev, 0) : e1;
            if (e == cudaSuccess) e = e2;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e3 = cudaStreamEndCapture(b->cap, &g);
        if (st != SONAR_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(ctx, e, "graph fork"); }
        CU(e3, "graph capture");
        b->step_kernels = kernel_nodes(g);
        const cudaError_t e4 = cudaGraphInstantiate(&b->step, g, 0);
        cudaGraphDestroy(g);
        CU(e4, "graph instantiation");
        b->step_key = key;
        ++b->graphs;
    }
    CU(cudaGraphLaunch(b->step, (cudaStream_t)stream), "graph launch");
    b->ran_fwd = b->ran_bwd = true;
    return SONAR_OK;
}

extern "C" sonar_status sonar_batch_info(sonar_batch_t b, int64_t out[5]) {
    if (!b || !out) return SONAR_ERR_ARG;
    int64_t rays = 0;
    for (const SensorDev& S : b->hs) rays += (int64_t)S.nb * S.ne;
    out[0] = (int64_t)b->units.size();
    out[1] = rays;
    out[2] = persistent_grid(b, 1);
    out[3] = b->block;
    out[4] = b->graphs;
    return SONAR_OK;
}

extern "C" sonar_status sonar_batch_kernels(sonar_batch_t b, int32_t out[2]) {
    if (!b || !out) return SONAR_ERR_ARG;
    out[0] = b->lean_last ? (b->fwd_lean ? b->fwd_lean_kernels : 0) : (b->fwd ? b->fwd_kernels : 0);
    out[1] = b->bwd ? b->bwd_kernels : 0;
    return SONAR_OK;
}

extern "C" sonar_status sonar_batch_timings(sonar_batch_t b, float ms[5]) {
    if (!b || !ms) return SONAR_ERR_ARG;
    sonar_ctx* ctx = b->ctx;
    for (int k = 0; k < 5; ++k) ms[k] = -1.0f;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (b->ran_fwd) {
        CU(cudaEventSynchronize(b->ev[2]), "cudaEventSynchronize");
        CU(cudaEventElapsedTime(&ms[0], b->ev[0], b->ev[6]), "cudaEventElapsedTime");
        CU(cudaEventElapsedTime(&ms[1], b->ev[6], b->ev[1]), "cudaEventElapsedTime");
        CU(cudaEventElapsedTime(&ms[2], b->ev[1], b->ev[2]), "cudaEventElapsedTime");
    }
    if (b->ran_bwd) {
        CU(cudaEventSynchronize(b->ev[5]), "cudaEventSynchronize");
        CU(cudaEventElapsedTime(&ms[3], b->ev[3], b->ev[4]), "cudaEventElapsedTime");
        CU(cudaEventElapsedTime(&ms[4], b->ev[4], b->ev[5]), "cudaEventElapsedTime");
    }
    return SONAR_OK;
}

extern "C" sonar_status sonar_batch_destroy(sonar_batch_t b) {
    if (!b) return SONAR_OK;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    batch_free_device(b);
    for (cudaEvent_t& e : b->ev)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
        if (b->h_stage_sc[k]) cudaFreeHost(b->h_stage_sc[k]);
        if (b->stage_ev[k]) cudaEventDestroy(b->stage_ev[k]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->join_ev) cudaEventDestroy(b->join_ev);
    delete b;
    return SONAR_OK;
}

// ===========================================================================
// autotuner
// ===========================================================================

namespace {

// Times the batch's forward launches, and its adjoint launches when `grad` is
// given (no graph): the best over `rounds` of the mean of `reps` back-to-back
// passes, after one warm-up pass; 1e30 when a launch sequence fails.
float time_batch(sonar_batch* b, const sonar_params* p, const float* d_theta, int32_t n_mat,
                 const sonar_batch_outputs* out, const float* grad, float* dtheta, cudaStream_t s, int reps,
                 int rounds) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bool ok = true;
    auto pass = [&] {
        ok = ok && batch_forward_launches(b, p, d_theta, n_mat, out, s) == SONAR_OK;
        if (grad)
            ok = ok && batch_backward_launches(b, p, d_theta, n_mat, grad, out->noised, out->hits, dtheta, s) ==
                           SONAR_OK;
    };
    pass();
    float best = 1e30f;
    for (int k = 0; k < rounds && ok; ++k) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) pass();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms / reps);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? best : 1e30f;   // a candidate whose launches failed is never chosen
}

}  // namespace

extern "C" sonar_status sonar_autotune(sonar_batch_t b, const sonar_params* p, const float* d_theta, int32_t n_mat,
                                       const sonar_batch_outputs* out, void* stream) {
    if (!b) return SONAR_ERR_ARG;
    sonar_ctx* ctx = b->ctx;
    sonar_status st = check_params(ctx, p);
    if (st) return st;
    if (!d_theta || !out || !out->polar) return fail(ctx, SONAR_ERR_ARG, "NULL theta or outputs");
    for (const sonar_batch_item& it : b->items)
        if ((st = check_scene(ctx, it.scene_id)) || (st = check_nmat(ctx, it.scene_id, n_mat))) return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    CU(batch_scratch(b, out), "batch scratch");
    std::vector<ShapeKey> shapes;
    for (const sonar_batch_item& it : b->items) {
        const ShapeKey k{it.sensor.n_beams, it.sensor.n_elev, it.sensor.n_range_bins, it.sensor.n_az_bins};
        if (std::find(shapes.begin(), shapes.end(), k) == shapes.end()) shapes.push_back(k);
    }
    const std::vector<sonar_batch_item> all = b->items;
    // an upstream gradient for timing the adjoint: every element the float
    // with bytes 0x3A (about 7e-4)
    float* adj_grad = nullptr;
    float* adj_dtheta = nullptr;
    if (out->hits && out->noised) {
        if (cudaMalloc(&adj_grad, sizeof(float) * std::max<int64_t>(1, b->total_polar)) != cudaSuccess ||
            cudaMalloc(&adj_dtheta, sizeof(float) * (n_mat + 2)) != cudaSuccess ||
            cudaMemsetAsync(adj_grad, 0x3A, sizeof(float) * std::max<int64_t>(1, b->total_polar), s) != cudaSuccess) {
            if (adj_grad) cudaFree(adj_grad);
            if (adj_dtheta) cudaFree(adj_dtheta);
            return fail(ctx, SONAR_ERR_OOM, "autotune scratch");
        }
    }
    // per shape, timed on that shape's items alone
    for (const ShapeKey& k : shapes) {
        std::vector<sonar_batch_item> sub;
        for (const sonar_batch_item& it : all)
            if (ShapeKey{it.sensor.n_beams, it.sensor.n_elev, it.sensor.n_range_bins, it.sensor.n_az_bins} == k)
                sub.push_back(it);
        b->items = sub;
        Tune best;
        best.block = 128;
        float best_ms = 1e30f;
        // the trace warp tile (beams x elevations per warp) and register budget,
        // with default binning shapes
        for (int occ : {0, kTraceCap, kTraceWide, kTraceCap | kTraceWide}) {
            for (int tb : {1, 2, 4, 8, 16, 32}) {
                ctx->tune[k] = Tune{0, tb, 128, occ};
                if ((st = batch_plan(b)) != SONAR_OK) goto restore;
                if (batch_scratch(b, out) != cudaSuccess) { st = fail(ctx, SONAR_ERR_OOM, "batch scratch"); goto restore; }
                const float ms = time_batch(b, p, d_theta, n_mat, out, nullptr, nullptr, s, 3, 3);
                if (cudaGetLastError() != cudaSuccess) continue;
                if (ms < best_ms) { best_ms = ms; best.tb = tb; best.occ = occ; }
            }
        }
        // then columns per binning unit and the binning block size (which also
        // sets the adjoint's block and ray chunks): forward and, when the caller's
        // outputs hold the hit records and I~, the adjoint of a constant
        // upstream gradient too
        best_ms = 1e30f;
        const int tb = best.tb, occ = best.occ;
        for (int block : {64, 128, 256}) {
            for (int cols : {1, 2, 4, 8, 16, 32}) {
                if (cols > k[3] || (size_t)cols * k[2] * 4 * 65 > kMaxDynSmem * 32) continue;
                ctx->tune[k] = Tune{cols, tb, block, occ};
                if ((st = batch_plan(b)) != SONAR_OK) goto restore;
                if (batch_scratch(b, out) != cudaSuccess) { st = fail(ctx, SONAR_ERR_OOM, "batch scratch"); goto restore; }
                const float* g = nullptr;
                if (adj_grad) {
                    if (cudaMalloc(&b->d_partials, sizeof(double) * b->adj_units.size() * (n_mat + 2)) != cudaSuccess) {
                        st = fail(ctx, SONAR_ERR_OOM, "batch scratch");
                        goto restore;
                    }
                    b->n_mat_cap = n_mat;
                    g = adj_grad;
                }
                const float ms = time_batch(b, p, d_theta, n_mat, out, g, adj_dtheta, s, 3, 3);
                if (cudaGetLastError() != cudaSuccess) continue;
                if (ms < best_ms) { best_ms = ms; best = Tune{cols, tb, block, occ}; }
            }
        }
        ctx->tune[k] = best;
    }
restore:
    b->items = all;
    if (adj_grad) cudaFree(adj_grad);
    if (adj_dtheta) cudaFree(adj_dtheta);
    {
        const sonar_status st2 = batch_plan(b);
        if (st == SONAR_OK) st = st2;
    }
    CU(cudaStreamSynchronize(s), "autotune synchronisation");
    return st;
}

extern "C" sonar_status sonar_tune_get(sonar_ctx_t ctx, int32_t* rows, int32_t cap, int32_t* count) {
    if (!ctx || !count) return SONAR_ERR_ARG;
    int k = 0;
    for (auto& kv : ctx->tune) {
        if (rows && k < cap) {
            int32_t* r = rows + 8 * k;
            r[0] = kv.first[0]; r[1] = kv.first[1]; r[2] = kv.first[2]; r[3] = kv.first[3];
            r[4] = kv.second.cols; r[5] = kv.second.tb; r[6] = kv.second.block; r[7] = kv.second.occ;
        }
        ++k;
    }
    *count = k;
    return SONAR_OK;
}

extern "C" sonar_status sonar_tune_set(sonar_ctx_t ctx, const int32_t* rows, int32_t count) {
    if (!ctx || (!rows && count > 0) || count < 0) return fail(ctx, SONAR_ERR_ARG, "bad tune rows");
    for (int k = 0; k < count; ++k) {
        const int32_t* r = rows + 8 * k;
        if (r[0] < 1 || r[1] < 1 || r[2] < 1 || r[3] < 1 || r[4] < 1 || r[5] < 1 || r[5] > 32 ||
            (r[5] & (r[5] - 1)) || r[6] < 32 || r[6] > 512 || (r[6] & 31) || (r[7] & ~(kTraceCap | kTraceWide)))
            return fail(ctx, SONAR_ERR_ARG, "bad tune row " + std::to_string(k));
        ctx->tune[ShapeKey{r[0], r[1], r[2], r[3]}] = Tune{r[4], r[5], r[6], r[7]};
    }
    return SONAR_OK;
}

// ===========================================================================
// counters
// ===========================================================================

extern "C" sonar_status sonar_uw_image(sonar_ctx_t ctx, const float* d_J, const float* d_depth, int64_t n_pixels,
                                       const float coef[9], float* d_I, void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    if (n_pixels < 0) return fail(ctx, SONAR_ERR_ARG, "n_pixels < 0");
    if (!coef) return fail(ctx, SONAR_ERR_ARG, "coef is NULL");
    for (int c = 0; c < 9; ++c) {
        if (!std::isfinite(coef[c])) return fail(ctx, SONAR_ERR_ARG, "coefficients must be finite");
        if (c < 6 && coef[c] < 0.0f) return fail(ctx, SONAR_ERR_ARG, "attenuation and backscatter must be >= 0");
    }
    if (n_pixels == 0) return SONAR_OK;
    if (!d_J || !d_depth || !d_I) return fail(ctx, SONAR_ERR_ARG, "NULL image buffer");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    UwCoef k;
    for (int c = 0; c < 3; ++c) {
        k.b_attn[c] = coef[c];
        k.b_bs[c] = coef[3 + c];
        k.b_inf[c] = coef[6 + c];
    }
    CU(launch_uw_image(d_J, d_depth, n_pixels, k, d_I, ctx->sm_count, (cudaStream_t)stream), "image launch");
    return SONAR_OK;
}

extern "C" sonar_status sonar_dvl(sonar_ctx_t ctx, int32_t scene_id, const float* d_poses, const float* d_vel,
                                  int64_t n, const sonar_dvl_params* p, uint64_t seed, float* d_ranges,
                                  float* d_vel_out, int32_t* d_flags, float* d_period, void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    if (!p) return fail(ctx, SONAR_ERR_ARG, "params is NULL");
    if (n < 0) return fail(ctx, SONAR_ERR_ARG, "n < 0");
    sonar_status st;
    if ((st = check_scene(ctx, scene_id))) return st;
    const float vals[] = {p->tilt, p->r_min, p->r_max, p->sigma_b, p->t0, p->t1, p->t_lost};
    for (float v : vals)
        if (!std::isfinite(v)) return fail(ctx, SONAR_ERR_ARG, "DVL parameters must be finite");
    if (!(p->tilt > 0.0f && p->tilt < 1.5707963f)) return fail(ctx, SONAR_ERR_ARG, "tilt must lie in (0, pi/2)");
    if (!(p->r_min >= 0.0f && p->r_max > p->r_min)) return fail(ctx, SONAR_ERR_ARG, "need 0 <= r_min < r_max");
    if (p->min_beams != 3 && p->min_beams != 4) return fail(ctx, SONAR_ERR_ARG, "min_beams must be 3 or 4");
    if (p->sigma_b < 0.0f || p->t0 < 0.0f || p->t1 < 0.0f || !(p->t_lost > 0.0f))
        return fail(ctx, SONAR_ERR_ARG, "need sigma_b, t0, t1 >= 0 and t_lost > 0");
    if (n == 0) return SONAR_OK;
    if (!d_poses || !d_vel || !d_ranges || !d_vel_out || !d_flags || !d_period)
        return fail(ctx, SONAR_ERR_ARG, "NULL buffer");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    DvlArgs a{};
    a.scene = scene_dev(ctx->scenes[scene_id]);
    a.pose = d_poses;
    a.vel_world = d_vel;
    a.n = n;
    for (int k = 0; k < 4; ++k) {
        const double az = M_PI / 4.0 + k * (M_PI / 2.0);
        a.beam[k][0] = (float)(std::sin((double)p->tilt) * std::cos(az));
        a.beam[k][1] = (float)(std::sin((double)p->tilt) * std::sin(az));
        a.beam[k][2] = (float)(-std::cos((double)p->tilt));
    }
    a.r_min = p->r_min;
    a.r_max = p->r_max;
    a.sigma_b = p->sigma_b;
    a.t0 = p->t0;
    a.t1 = p->t1;
    a.t_lost = p->t_lost;
    a.min_beams = p->min_beams;
    a.seed_lo = (uint32_t)seed;
    a.seed_hi = (uint32_t)(seed >> 32);
    a.ranges = d_ranges;
    a.vel = d_vel_out;
    a.flags = d_flags;
    a.period = d_period;
    a.err = ctx->d_err;
    CU(launch_dvl(a, (cudaStream_t)stream), "DVL launch");
    return SONAR_OK;
}

extern "C" sonar_status sonar_dvl_schedule(sonar_ctx_t ctx, const float* d_period, int64_t n_veh, int64_t n_steps,
                                           float dt, int32_t* d_emit, void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    if (n_veh < 0 || n_steps < 0) return fail(ctx, SONAR_ERR_ARG, "negative count");
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(ctx, SONAR_ERR_ARG, "dt must be finite and > 0");
    if (n_veh == 0 || n_steps == 0) return SONAR_OK;
    if (!d_period || !d_emit) return fail(ctx, SONAR_ERR_ARG, "NULL buffer");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    CU(launch_dvl_schedule(d_period, n_veh, n_steps, dt, d_emit, (cudaStream_t)stream), "DVL schedule launch");
    return SONAR_OK;
}

extern "C" sonar_status sonar_trace_stats(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                                          const sonar_params* params, void* stream, int64_t out[6]) {
    if (!ctx || !out) return fail(ctx, SONAR_ERR_ARG, "NULL argument");
    sonar_status st;
    if ((st = check_scene(ctx, scene_id)) || (st = check_sensor(ctx, sensor)) || (st = check_params(ctx, params)))
        return st;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const SceneStore& sc = ctx->scenes[scene_id];
    const int64_t node_words = sc.n_pairs / 32 + 1, tri_words = sc.n_tris / 32 + 1;
    unsigned long long* cnt = nullptr;
    uint32_t *nb = nullptr, *tb = nullptr;
    CU(cudaMalloc(&cnt, sizeof(unsigned long long) * 8), "stats allocation");
    cudaError_t e = cudaMalloc(&nb, sizeof(uint32_t) * node_words);
    if (e == cudaSuccess) e = cudaMalloc(&tb, sizeof(uint32_t) * tri_words);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nb, 0, sizeof(uint32_t) * node_words, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb, 0, sizeof(uint32_t) * tri_words, s);
    TraceCounters tc{cnt, cnt + 1, cnt + 2, nb, tb};
    // the tuned warp tiles of this sensor shape: a lane's visits depend a little
    // on its warp's rays (leaves are parked until the whole warp holds one)
    const Tune t = tune_for(ctx, *sensor);
    SensorDev S = make_sensor(*sensor, 0, 0, t, 0, 0);
    float4* trig = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&trig, sizeof(float4) * (S.nb + S.ne));
    S.trig = trig;
    if (e == cudaSuccess) e = launch_trig(nullptr, S, 1, S.nb + S.ne, s);
    if (e == cudaSuccess) e = launch_stats(S, scene_dev(sc), *params, tc, ctx->d_err, s);
    if (e == cudaSuccess) e = launch_popcount(nb, node_words, cnt + 3, s);
    if (e == cudaSuccess) e = launch_popcount(tb, tri_words, cnt + 4, s);
    unsigned long long h[8] = {};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    cudaFree(nb);
    cudaFree(tb);
    cudaFree(trig);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace statistics");
    out[0] = (int64_t)h[0];
    out[1] = (int64_t)h[1];
    out[2] = (int64_t)h[3];
    out[3] = (int64_t)h[4];
    out[4] = (int64_t)S.nb * S.ne;
    out[5] = (int64_t)h[2];
    return SONAR_OK;
}

extern "C" sonar_status sonar_philox(sonar_ctx_t ctx, const uint32_t* d_counters, int64_t n, uint64_t seed,
                                     uint32_t* d_out, void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    if (n < 0) return fail(ctx, SONAR_ERR_ARG, "n < 0");
    if (n == 0) return SONAR_OK;
    if (!d_counters || !d_out) return fail(ctx, SONAR_ERR_ARG, "NULL buffer");
    if (!aligned16(d_counters) || !aligned16(d_out)) return fail(ctx, SONAR_ERR_ARG, "buffers must be 16-byte aligned");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    CU(launch_philox(d_counters, n, (uint32_t)seed, (uint32_t)(seed >> 32), d_out, (cudaStream_t)stream),
       "philox launch");
    return SONAR_OK;
}

extern "C" sonar_status sonar_probe_l2_read(sonar_ctx_t ctx, const void* d_buf, int64_t bytes, int32_t passes,
                                            float* d_block_sums, int32_t n_blocks, void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    if (!d_buf || !d_block_sums) return fail(ctx, SONAR_ERR_ARG, "NULL buffer");
    if (bytes <= 0 || bytes % 16 != 0) return fail(ctx, SONAR_ERR_ARG, "bytes must be a positive multiple of 16");
    if (reinterpret_cast<uintptr_t>(d_buf) % 16 != 0) return fail(ctx, SONAR_ERR_ARG, "buffer not 16-byte aligned");
    if (passes < 1) return fail(ctx, SONAR_ERR_ARG, "passes < 1");
    if (n_blocks < 1 || n_blocks > 65535) return fail(ctx, SONAR_ERR_ARG, "n_blocks outside [1, 65535]");
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    CU(launch_l2_read(d_buf, bytes, passes, d_block_sums, n_blocks, (cudaStream_t)stream), "probe launch");
    return SONAR_OK;
}

// ===========================================================================
// rendering without device allocation
// ===========================================================================

namespace {

// The scratch of sonar_render_noalloc: a fixed array in the library's device
// image, resident on every device that loads the library until the process
// exits.  Host code cannot use the symbol as a pointer; each device's address
// comes from cudaGetSymbolAddress.
static __device__ __align__(256) float g_noalloc_scratch[SONAR_NOALLOC_SCRATCH_WORDS];

std::mutex g_noalloc_mutex;
std::map<unsigned long long, void*> g_noalloc_addr;   // by context id (unique for the process)

// The unique id of the calling thread's current context (cuCtxGetCurrent and
// cuCtxGetId, through the runtime's driver entry points); false when the
// driver does not offer them.
bool current_context_id(unsigned long long* id) {
    typedef int (*get_current_t)(void**);
    typedef int (*get_id_t)(void*, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        void* g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (get_current_t)f;
            get_id = (get_id_t)g;
        }
        looked_up = true;
    }
    void* ctx = nullptr;
    return get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current context (the caller has
// made the context's device current).  Looked up once per context: a context
// that is destroyed and created again (cudaDeviceReset) reloads the library's
// device code, the array may move, and the new context has a new id.  Where
// the driver cannot name the context, the address is looked up on every call
// (a host-side lookup once the device code is loaded).
cudaError_t noalloc_scratch(void** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    const bool keyed = current_context_id(&id);
    if (keyed) {
        auto it = g_noalloc_addr.find(id);
        if (it != g_noalloc_addr.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (keyed) g_noalloc_addr[id] = p;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" sonar_status sonar_render_noalloc(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                                             const sonar_params* params, const float* d_theta, int32_t n_mat,
                                             uint64_t seed, uint64_t frame, const sonar_outputs* out,
                                             void* stream) {
    if (!ctx) return SONAR_ERR_ARG;
    sonar_status st;
    if ((st = check_scene(ctx, scene_id)) || (st = check_sensor(ctx, sensor)) || (st = check_params(ctx, params)) ||
        (st = check_nmat(ctx, scene_id, n_mat)))
        return st;
    if (!d_theta) return fail(ctx, SONAR_ERR_ARG, "d_theta is NULL");
    if (!out || !out->polar) return fail(ctx, SONAR_ERR_ARG, "outputs or outputs->polar is NULL");
    if (out->hits && !aligned16(out->hits)) return fail(ctx, SONAR_ERR_ARG, "hits must be 16-byte aligned");
    if (out->fan && (out->fan_w < 1 || out->fan_h < 1)) return fail(ctx, SONAR_ERR_ARG, "fan size must be >= 1");
    // scratch layout (words): the image maximum at 0; from 64 the exact-ray
    // tables (4 words a beam and an elevation); then, each at a 256-byte
    // boundary, the hit records (4 words a ray) and the noised image unless the
    // caller passes them
    const int64_t npol = (int64_t)sensor->n_range_bins * sensor->n_az_bins;
    const int64_t trig_words = 4 * ((int64_t)sensor->n_beams + sensor->n_elev);
    const int64_t hits_at = 64 + (trig_words + 63) / 64 * 64;
    const int64_t hit_words = out->hits ? 0 : 4 * (int64_t)sensor->n_beams * sensor->n_elev;
    const int64_t noised_at = hits_at + (hit_words + 63) / 64 * 64;
    const int64_t need = out->noised ? noised_at : noised_at + npol;
    if (need > (int64_t)SONAR_NOALLOC_SCRATCH_WORDS)
        return fail(ctx, SONAR_ERR_ARG, "sonar_render_noalloc: frame needs " + std::to_string(need) +
                                            " scratch words, the fixed scratch holds " +
                                            std::to_string(SONAR_NOALLOC_SCRATCH_WORDS) +
                                            " (pass outputs->hits and outputs->noised to need fewer)");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    void* base = nullptr;
    CU(noalloc_scratch(&base), "cudaGetSymbolAddress of the fixed scratch");
    uint32_t* rowmax = (uint32_t*)base;
    sonar_hit* hits = out->hits ? out->hits : (sonar_hit*)((float*)base + hits_at);
    float* noised = out->noised ? out->noised : (float*)base + noised_at;
    const Tune t = single_tune(ctx, *sensor);
    SensorDev S = make_sensor(*sensor, seed, frame, t, out->fan ? out->fan_w : 0, out->fan ? out->fan_h : 0);
    S.trig = (float4*)((float*)base + 64);
    // single_forward clears the maximum (the array still holds the previous
    // call's values); hit records and the noised image are fully overwritten
    st = single_forward(ctx, S, scene_dev(ctx->scenes[scene_id]), params, d_theta, n_mat, hits, noised, out->binned,
                        rowmax, t.block, s);
    if (st != SONAR_OK) return st;
    return single_post(ctx, S, params->normalise, noised, rowmax, out->polar, out->fan, s);
}
