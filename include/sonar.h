/*
 * sonar.h -- C ABI of libsonar: forward-looking imaging-sonar rendering on one
 * GB300 (sm_103a).
 *
 * Method: OceanSim (arXiv 2503.01074), Sec. III-A-2.  Each (beam, elevation)
 * sample of the sonar field of view casts one ray into a triangle scene; a
 * return scores mu[m] * cos * exp(-2 alpha r) * gain (Eq. 2 in its two-way
 * form: the paper's alpha equals 2 alpha here); returns are summed into a
 * range x azimuth polar grid; additive Rayleigh and multiplicative Gaussian
 * noise are applied per bin (Eq. 3-6); each range row is normalised
 * (range-wise normalisation, end of Sec. III-A-2); the polar image is
 * resampled into a Cartesian fan image (the "plot styles" of the same
 * paragraph).  The gradient entry points are an addition: the analytic
 * adjoint of that pipeline with respect to (alpha, gain, mu).
 *
 * Conventions for every entry point
 *  - Pointers named d_* are DEVICE pointers on the context's GPU, owned by
 *    the caller and borrowed for the call; all others are host pointers read
 *    before the call returns.
 *  - Every call that takes a stream only enqueues work on it (cudaStream_t
 *    passed as void*; 0 = the legacy default stream); outputs are valid once
 *    that stream has reached the call.  No call aborts, traps or prints.
 *  - Argument errors are detected on the host before anything is enqueued and
 *    return SONAR_ERR_ARG; sonar_last_error() then holds a message.
 *  - Kernels that detect a fault (a traversal stack overflow, an index out of
 *    range) set a sticky device error word instead of trapping;
 *    sonar_check(ctx) synchronises and reports it as SONAR_ERR_DEVICE, then
 *    clears it.
 *  - A context is used by one host thread at a time, and its calls are
 *    stream-ordered: the context's own scratch (outputs passed as NULL, the
 *    single-sensor calls' exact-ray tables, which are rebuilt only when the
 *    angular geometry changes) is reused from call to call, so calls on
 *    different streams need the caller's synchronisation between them.
 *
 * World frame: z up.  Sensor frame: +y forward, +x right, +z up.  Ray (i, j)
 * of beam i in [0, n_beams) and elevation j in [0, n_elev) has azimuth
 * phi_i = -hfov/2 + (i + 1/2) hfov / n_beams and elevation
 * theta_j = -vfov/2 + (j + 1/2) vfov / n_elev; its sensor-frame direction is
 * (sin phi cos theta, cos phi cos theta, sin theta), rotated by `rot`.  The
 * canonical ray index is k = i * n_elev + j.
 */
#ifndef SONAR_H
#define SONAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sonar_ctx* sonar_ctx_t;
typedef struct sonar_batch* sonar_batch_t;

typedef enum {
    SONAR_OK = 0,
    SONAR_ERR_ARG = 1,      /* invalid argument; nothing was enqueued */
    SONAR_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    SONAR_ERR_OOM = 3,      /* device allocation failed */
    SONAR_ERR_TIMEOUT = 4,  /* reserved: no call returns it (no kernel waits on another) */
    SONAR_ERR_DEVICE = 5,   /* the sticky device error word was set */
    SONAR_ERR_STATE = 6     /* call not valid in the object's current state */
} sonar_status;

/* Sticky device error bits (sonar_check reports their OR in *bits). */
#define SONAR_DEVERR_STACK 0x1u    /* BVH traversal stack overflow */
#define SONAR_DEVERR_INDEX 0x2u    /* an index read from memory was out of range */
#define SONAR_DEVERR_TIMEOUT 0x4u  /* reserved: never set (no kernel spin-waits) */

/* Sonar geometry and pose.  rot is the sensor->world rotation, row-major:
 * d_world[a] = sum_b rot[3a + b] d_sensor[b].  hfov, vfov in radians, in
 * (0, pi]; 0 <= r_min < r_max in metres.  Range bin b_r covers
 * [r_min + b_r dr, r_min + (b_r + 1) dr), dr = (r_max - r_min) / n_range_bins;
 * azimuth bin b_a covers [-hfov/2 + b_a da, -hfov/2 + (b_a + 1) da),
 * da = hfov / n_az_bins.  Ray (i, j) falls into azimuth bin
 * floor((2i + 1) n_az_bins / (2 n_beams)). */
typedef struct {
    float pos[3];
    float rot[9];
    int32_t n_beams, n_elev, n_range_bins, n_az_bins;
    float hfov, vfov;
    float r_min, r_max;
} sonar_sensor;

/* Non-differentiable configuration. */
typedef struct {
    float sigma_sa;      /* Rayleigh scale of the additive noise (Eq. 3-4), >= 0 */
    float sigma_sm;      /* std deviation of the multiplicative noise (Eq. 5-6), >= 0 */
    float sigma_phi;     /* beam-pattern width in Eq. 3 (rad^2), > 0 */
    int32_t normalise;   /* 0 none, 1 range-row maximum (default), 2 global maximum */
    int32_t two_sided;   /* 1: incidence factor |d.n| (default); 0: max(0, -d.n) */
    int32_t clip_tmax;   /* 1: the cast ends at the sonar's maximum range, so only
                               returns with r < r_max are found (default); 0: the
                               cast is unbounded and records returns beyond r_max
                               too.  The images and gradients are the same either
                               way (returns at or beyond r_max are never binned);
                               the bounded cast visits fewer nodes. */
    int32_t accumulate;  /* 0: deterministic fold of each bin's returns in canonical
                               ray order (default; bitwise reproducible);
                            1: warp-aggregated shared-memory atomics */
    int32_t reserved;
} sonar_params;

/* Per-ray hit record, 16 bytes, indexed by the canonical ray index.
 * key = b_r * n_az_bins + b_a, or 0xFFFFFFFF if the return is not binned
 * (miss, or r outside [r_min, r_max)); tri = the caller's triangle index, or
 * 0xFFFFFFFF on a miss; r = hit range in metres (+inf on a miss);
 * cos = the incidence factor used in the score (0 on a miss). */
typedef struct {
    uint32_t key;
    uint32_t tri;
    float r;
    float cos;
} sonar_hit;

/* Outputs of one render.  polar is required; the rest may be NULL.
 *   polar   [n_range_bins][n_az_bins] f32: the normalised image N
 *   noised  [n_range_bins][n_az_bins] f32: I~ after Eq. 5, before normalisation
 *           (the backward pass needs it)
 *   binned  [n_range_bins][n_az_bins] f32: P, the summed intensities before noise
 *   hits    [n_beams * n_elev] sonar_hit
 *   fan     [fan_h][fan_w] f32 (row 0 = far edge), requires fan_w, fan_h > 0 */
typedef struct {
    float* polar;
    float* noised;
    float* binned;
    sonar_hit* hits;
    float* fan;
    int32_t fan_w, fan_h;
} sonar_outputs;

/* Library version and build information (static string). */
const char* sonar_version(void);

/* Creates a context on CUDA device `device` (which becomes current for the
 * calling thread).  *out receives the handle. */
sonar_status sonar_create(int32_t device, sonar_ctx_t* out);

/* Synchronises the device, frees every scene, batch and scratch buffer the
 * context owns.  NULL is accepted. */
sonar_status sonar_destroy(sonar_ctx_t ctx);

/* Message describing the last failed call on this context (static storage
 * owned by the context; "" if none).  ctx may be NULL for creation errors. */
const char* sonar_last_error(sonar_ctx_t ctx);

/* Synchronises the device and reports the sticky device error word:
 * SONAR_ERR_DEVICE if any bit was set (bits in *bits if non-NULL), after
 * which the word is cleared. */
sonar_status sonar_check(sonar_ctx_t ctx, uint32_t* bits);

/* Builds the scene's bounding-volume hierarchy (the geometry query of
 * Sec. III-A-2: Morton codes, radix sort, Karras hierarchy, bottom-up box
 * refit, node packing).  d_verts [n_verts][3] f32, d_tris [n_tris][3] int32
 * vertex indices, d_mat [n_tris] int32 material ids >= 0 (the reflectivity
 * A_r of Eq. 2 per semantic class).  The inputs are read during the call and
 * not retained.  Validates indices and vertex finiteness (synchronises the
 * stream once).  n_tris may be 0 (every ray misses) and must be < 2^28 - 2.
 * *scene_id receives the handle used by the render calls. */
sonar_status sonar_scene_upload(sonar_ctx_t ctx, const float* d_verts, int64_t n_verts,
                                const int32_t* d_tris, const int32_t* d_mat, int64_t n_tris,
                                void* stream, int32_t* scene_id);

/* Releases a scene (synchronises the device first). */
sonar_status sonar_scene_release(sonar_ctx_t ctx, int32_t scene_id);

/* Scene statistics: out[0] triangles, out[1] nodes of the 4-wide tree, out[2]
 * binary tree height, out[3] maximum material id, out[4] device bytes held
 * (both trees and the triangles). */
sonar_status sonar_scene_info(sonar_ctx_t ctx, int32_t scene_id, int64_t out[5]);

/* One sonar frame (Sec. III-A-2): ray cast, intensity (Eq. 2), polar
 * binning, noise (Eq. 3-6) with Philox4x32-10 keyed by `seed`, counter
 * (bin, frame lo32, 0, frame hi32), range-wise normalisation and, if
 * out->fan is set, the fan image.
 * d_theta [2 + n_mat] f32 = (alpha, gain, mu[0], ..., mu[n_mat - 1]);
 * n_mat must exceed the scene's largest material id, 1 <= n_mat <= 1024. */
sonar_status sonar_render(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                          const sonar_params* params, const float* d_theta, int32_t n_mat,
                          uint64_t seed, uint64_t frame, const sonar_outputs* out,
                          void* stream);

/* Maximum scratch, in 4-byte words, that sonar_render_noalloc can use: 64
 * words, plus 4 words a beam and an elevation (exact-ray tables), plus 4 words
 * a ray for the hit records when out->hits is NULL, plus n_range_bins *
 * n_az_bins words for the noised image when out->noised is NULL (each part
 * rounded up to 64 words). */
#define SONAR_NOALLOC_SCRATCH_WORDS (1u << 20)

/* sonar_render for callers that must not allocate device memory: a render
 * loop with a fixed memory budget whose device memory is all owned by its
 * own pool, or real-time code where an allocation could block or
 * synchronise the device.  This call makes no allocation of any kind: its
 * scratch is a fixed array of SONAR_NOALLOC_SCRATCH_WORDS words (4 MiB)
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.  The caller still provides every input and
 * output, as for sonar_render, and gets the same results.
 *   - A frame needing more scratch than the array holds is rejected with
 *     SONAR_ERR_ARG before anything is enqueued (pass out->hits and
 *     out->noised to need only the small fixed parts).
 *   - The first call on a device looks up the array's device address (which
 *     may load the library's device code) and caches it for that device's
 *     current context; make that first call before any stream capture on
 *     that device.  After cudaDeviceReset the next call is a first call again
 *     (the new context loads the device code anew and the array may move).
 *   - All calls on a device share the one array, and it keeps the last
 *     call's contents (each call clears what it needs cleared): calls whose
 *     work can overlap on the GPU (different streams, or different contexts
 *     on the same device) race on it and must be serialised by the caller.
 * The paper has no counterpart of this entry point. */
sonar_status sonar_render_noalloc(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                                  const sonar_params* params, const float* d_theta, int32_t n_mat,
                                  uint64_t seed, uint64_t frame, const sonar_outputs* out,
                                  void* stream);

/* Resamples any polar image d_polar [n_range_bins][n_az_bins] into a fan
 * image d_fan [fan_h][fan_w]: square pixels, sensor at the bottom centre,
 * scale = min(fan_w / (2 r_max sin(hfov/2)), fan_h / r_max) pixels per metre;
 * bilinear over bin centres, clamped to the edge bins; 0 outside the fan. */
sonar_status sonar_fan_resample(sonar_ctx_t ctx, const sonar_sensor* sensor,
                                const float* d_polar, int32_t fan_w, int32_t fan_h,
                                float* d_fan, void* stream);

/* Adjoint of sonar_render.  d_grad_polar = dL/dN [n_range_bins][n_az_bins];
 * d_noised = the I~ that sonar_render wrote for the same (scene, sensor,
 * params, theta, seed, frame); d_hits = that render's hit records, or NULL to
 * recompute them by re-casting the rays into context scratch (bitwise the
 * same records).
 * Writes d_dtheta [2 + n_mat] f32 = (dL/dalpha, dL/dgain, dL/dmu[...]),
 * overwriting it.  Deterministic: the same inputs give the same bits. */
sonar_status sonar_render_backward(sonar_ctx_t ctx, int32_t scene_id,
                                   const sonar_sensor* sensor, const sonar_params* params,
                                   const float* d_theta, int32_t n_mat, uint64_t seed,
                                   uint64_t frame, const float* d_grad_polar,
                                   const float* d_noised, const sonar_hit* d_hits,
                                   float* d_dtheta, void* stream);

/* ---- batched rendering: many sensors, several scenes, one persistent launch ---- */

/* One sensor of a batch.  Offsets are element offsets into the packed output
 * buffers passed to sonar_render_batch (polar/noised/binned share
 * polar_offset; hits use hits_offset; the fan uses fan_offset).  fan_w,
 * fan_h = 0 skips the fan for this sensor. */
typedef struct {
    int32_t scene_id;
    int32_t fan_w, fan_h;
    int32_t reserved;
    sonar_sensor sensor;
    uint64_t seed, frame;
    int64_t polar_offset, hits_offset, fan_offset;
} sonar_batch_item;

/* Packed outputs of a batch; as sonar_outputs, with per-item offsets.
 * polar is required; others may be NULL (fan is skipped for every item if
 * NULL). */
typedef struct {
    float* polar;
    float* noised;
    float* binned;
    sonar_hit* hits;
    float* fan;
} sonar_batch_outputs;

/* Plans a batch: validates the items, splits every sensor into work units of
 * whole azimuth columns (shapes from the autotuner's cache when it has an
 * entry for the sensor shape, defaults otherwise), orders the units
 * largest-first for the persistent launch, and uploads the descriptors
 * (synchronous).  n_items >= 1. */
sonar_status sonar_batch_create(sonar_ctx_t ctx, const sonar_batch_item* items,
                                int32_t n_items, sonar_batch_t* out);

/* Replaces poses, seeds and frames (and scene ids, fields of view and range
 * windows) of a planned batch.  Item count, shapes (beams, elevations, bins,
 * fan size) and offsets must match the plan.  A shared fan coordinate table
 * is rebuilt by the next render once its owner's fan geometry has changed;
 * items whose geometry no longer matches their table's compute their own.  Enqueued on `stream` from
 * host staging memory owned by the batch; `items` may be reused at once. */
sonar_status sonar_batch_update(sonar_batch_t batch, const sonar_batch_item* items,
                                int32_t n_items, void* stream);

/* Renders every item of the batch: one launch builds the exact-ray sin/cos
 * tables, one casts every ray of every sensor, one persistent launch bins and
 * adds noise for all column work units (dynamic work list), one normalises
 * every range row, and the fans are resampled by one launch for the items
 * that share a fan geometry (after refreshing any coordinate table whose
 * geometry changed) and one for the others.  The first call for a given
 * (params, theta, outputs) captures the launches in a CUDA graph; later calls
 * with the same arguments replay it.  A call with no sonar_batch_update (and
 * no re-plan) since the last forward replays a second graph without the two
 * table launches, whose tables are then current (calls on one batch are
 * stream-ordered, as for a context).  Results per item equal sonar_render's
 * for the same item and tile shape (bitwise, in deterministic accumulation). */
sonar_status sonar_render_batch(sonar_batch_t batch, const sonar_params* params,
                                const float* d_theta, int32_t n_mat,
                                const sonar_batch_outputs* out, void* stream);

/* Adjoint of sonar_render_batch for the loss summed over items: d_grad_polar
 * and d_noised packed like the polar output, d_hits packed like the hit
 * output or NULL (the records are recomputed by the ray-cast kernel into the
 * batch's own scratch).  Writes d_dtheta [2 + n_mat], the gradient
 * summed over items.  Graph-captured like the forward. */
sonar_status sonar_render_batch_backward(sonar_batch_t batch, const sonar_params* params,
                                         const float* d_theta, int32_t n_mat,
                                         const float* d_grad_polar, const float* d_noised,
                                         const sonar_hit* d_hits, float* d_dtheta,
                                         void* stream);

/* One step of forward and adjoint for a caller whose upstream gradient is known
 * before the forward runs (a fixed target's sensitivity, a gradient image from
 * the caller's own pipeline): renders like sonar_render_batch into `out`, and
 * writes d_dtheta [2 + n_mat], the adjoint of d_grad_polar (packed like the
 * polar output) through this forward's I~ and hit records (out->noised and
 * out->hits, or the batch's scratch when NULL).  The adjoint needs I~ and the
 * records only, so one CUDA graph runs it beside the normalisation and fan
 * launches.  Results equal sonar_render_batch followed by
 * sonar_render_batch_backward with the same arguments (bitwise).  Captured once
 * per (params, theta, outputs, grad, dtheta) and replayed after. */
sonar_status sonar_render_batch_step(sonar_batch_t batch, const sonar_params* params,
                                     const float* d_theta, int32_t n_mat,
                                     const sonar_batch_outputs* out, const float* d_grad_polar,
                                     float* d_dtheta, void* stream);

/* Plan statistics: out[0] work units, out[1] total rays, out[2] persistent
 * grid size, out[3] block size, out[4] graphs captured so far. */
sonar_status sonar_batch_info(sonar_batch_t batch, int64_t out[5]);

/* Kernel launches per replay: out[0] kernel nodes of the forward graph replayed
 * last (with or without the table launches), out[1] of the current adjoint graph (0 for a graph not captured yet;
 * -1 if the graph could not be inspected); the step graph of
 * sonar_render_batch_step holds the kernels of both.  Host only, no
 * synchronisation. */
sonar_status sonar_batch_kernels(sonar_batch_t batch, int32_t out[2]);

/* Device durations, in milliseconds, of the phases of the most recent
 * sonar_render_batch and sonar_render_batch_backward replays (or of both
 * branches of a sonar_render_batch_step replay, where ms[3] and ms[4] overlap
 * ms[2]), measured by CUDA
 * events captured inside their graphs: ms[0] the ray-cast launch, ms[1] the
 * binning/noise launch, ms[2] the normalisation and fan launches, ms[3] the
 * adjoint row-term launch, ms[4] the adjoint gather and final-reduction
 * launches.  Waits for those replays to finish; a phase not yet run reports
 * -1. */
sonar_status sonar_batch_timings(sonar_batch_t batch, float ms[5]);

sonar_status sonar_batch_destroy(sonar_batch_t batch);

/* ---- autotuner ---- */

/* Times candidate tile shapes on the batch's own sensors and records the
 * fastest per sensor shape (n_beams, n_elev, n_range_bins, n_az_bins) in the
 * context's tuning cache; later sonar_batch_create and sonar_render calls use
 * it.  Stage 1 times the forward launches over the ray-cast warp tiles (beams
 * x elevations per warp) and register variants; stage 2 times the columns per
 * binning work unit and the block size, which also shape the adjoint, on the
 * forward launches plus, when `out` holds hit records and I~, the adjoint of
 * a constant upstream gradient.  Each candidate scores the best of 3 rounds
 * of 3 passes.  Runs on `stream` and synchronises it; allocates and frees its
 * own scratch (a polar-sized gradient).  Outputs of `out` are overwritten. */
sonar_status sonar_autotune(sonar_batch_t batch, const sonar_params* params,
                            const float* d_theta, int32_t n_mat,
                            const sonar_batch_outputs* out, void* stream);

/* Tuning cache entries: writes up to `cap` rows of 8 int32
 * (n_beams, n_elev, n_range_bins, n_az_bins, cols, tb, block, occ), tb =
 * beams per ray-cast warp (a power of two <= 32; elevations = 32 / tb), occ =
 * the ray-cast variant, a sum of flags: 8 caps its registers at 64 (32
 * one-warp blocks per SM), 16 walks the 8-wide tree instead of the 4-wide one
 * (both are built per scene; the hit records are the same either way).  A
 * batch takes the row's variant; a single-sensor call whose ray cast is at
 * most one wave of one-warp blocks (32 per SM) walks the 8-wide tree without
 * the register cap, and a larger one the 4-wide tree with its row's cap.
 * Returns the number of entries in *count. */
sonar_status sonar_tune_get(sonar_ctx_t ctx, int32_t* rows, int32_t cap, int32_t* count);

/* Adds or replaces cache entries (rows as above), e.g. loaded from a file. */
sonar_status sonar_tune_set(sonar_ctx_t ctx, const int32_t* rows, int32_t count);

/* ---- underwater camera image (Sec. III-A-1, Eq. 1) ---- */

/* Water-column effects on a camera image.  For every pixel k and colour
 * channel c (R, G, B):
 *   I_c = J_c exp(-beta_attn,c d) + B_inf,c (1 - exp(-beta_bs,c d)).
 * d_J      [n_pixels][3] f32, device: the in-air image J (pixel-major RGB).
 * d_depth  [n_pixels] f32, device: the depth d in metres (+inf where no
 *          geometry: the pixel then shows the veiling light).
 * coef     9 floats, host: beta_attn (R, G, B), beta_bs (R, G, B) in 1/m,
 *          finite and >= 0 (0 = no attenuation at any depth); B_inf (R, G, B),
 *          finite.
 * d_I      [n_pixels][3] f32, device, out; may be d_J itself (in place).
 * All buffers are the caller's; work is enqueued on `stream`.  16-byte aligned
 * buffers take a vectorised path.  Errors: SONAR_ERR_ARG (NULL buffer with
 * n_pixels > 0, n_pixels < 0, bad coefficient), before anything is enqueued. */
sonar_status sonar_uw_image(sonar_ctx_t ctx, const float* d_J, const float* d_depth, int64_t n_pixels,
                            const float coef[9], float* d_I, void* stream);

/* ---- DVL (Sec. III-A-3) ---- */

/* DVL configuration.  The paper describes a four-beam convex Janus array with
 * a range-dependent measurement rate and dropout, and fixes no numbers; these
 * are this library's readings, all adjustable:
 *   tilt       beam angle off the sensor's down axis (rad), in (0, pi/2);
 *              beam k points at azimuth 45 + 90 k degrees around that axis
 *   r_min, r_max  a beam is valid when its closest hit lies in [r_min, r_max] (m)
 *   min_beams  valid beams needed for a velocity (3 or 4)
 *   sigma_b    standard deviation of each beam's radial-velocity noise (m/s), >= 0
 *   t0, t1     ping period t0 + t1 * (farthest valid range) (s, s/m), >= 0
 *   t_lost     ping period while the velocity is invalid (s), > 0 */
typedef struct {
    float tilt, r_min, r_max;
    int32_t min_beams;
    float sigma_b, t0, t1, t_lost;
} sonar_dvl_params;

/* One DVL measurement for each of n poses against scene `scene_id`.
 * d_poses [n][12] f32: position (3) and sensor->world rotation (9, row-major;
 *   the sensor looks down its -z axis).  d_vel [n][3] f32: world velocity.
 * Each beam measures its radial velocity plus noise (Philox4x32-10, key =
 * seed, counter (pose lo, pose hi, 2, beam / 2); words 0, 1 -> even beams and
 * 2, 3 -> odd beams by the cosine branch of Box-Muller); the velocity is the
 * least-squares fit over the valid beams, in the sensor frame.
 * Out (device, caller-owned): d_ranges [n][4] closest-hit distance per beam
 * (+inf for a miss); d_vel_out [n][3] (0 when invalid); d_flags [n] (bit k:
 * beam k valid, bit 4: velocity valid); d_period [n] ping period (s).
 * Errors: SONAR_ERR_ARG for a bad scene, NULL buffer with n > 0, n < 0 or a
 * configuration outside the ranges above. */
sonar_status sonar_dvl(sonar_ctx_t ctx, int32_t scene_id, const float* d_poses, const float* d_vel, int64_t n,
                       const sonar_dvl_params* params, uint64_t seed, float* d_ranges, float* d_vel_out,
                       int32_t* d_flags, float* d_period, void* stream);

/* Measurement steps of n_veh vehicles simulated over n_steps steps of dt
 * seconds (d_period [n_veh][n_steps] from sonar_dvl on poses laid out vehicle
 * by vehicle): a measurement at step 0, then max(1, ceil(period / dt)) steps
 * after each one, the period read at that measurement.  d_emit [n_veh][n_steps]
 * int32 out: 1 at measurement steps, else 0.  Errors: SONAR_ERR_ARG for NULL
 * buffers with work to do, negative counts, dt <= 0 or not finite. */
sonar_status sonar_dvl_schedule(sonar_ctx_t ctx, const float* d_period, int64_t n_veh, int64_t n_steps, float dt,
                                int32_t* d_emit, void* stream);

/* ---- counters (roofline evidence) ---- */

/* Re-casts the rays of one sensor (with the warp tiles and the tree its
 * shape's tuning row names: 4-wide nodes of 128 bytes, or 8-wide ones of 256
 * bytes with variant flag 16) and counts node visits and triangle tests;
 * also marks every node and triangle touched.  out[0] node visits, out[1]
 * triangle tests, out[2] distinct nodes touched, out[3] distinct triangles
 * touched, out[4] rays, out[5] decisions taken exactly in float-float
 * arithmetic (uncertain FP32 tests and near ties).  Synchronises the stream. */
sonar_status sonar_trace_stats(sonar_ctx_t ctx, int32_t scene_id, const sonar_sensor* sensor,
                               const sonar_params* params, void* stream, int64_t out[6]);

/* The noise stream (Sec. III-A-2, Eq. 3-6 draws): Philox4x32-10 (Salmon et al.,
 * SC'11) of n counters under the key (seed lo 32 bits, seed hi 32 bits), by the
 * round function the render, adjoint and DVL kernels use.  A bin's draws come
 * from counter (bin index, frame lo, 0, frame hi): word 0 the Rayleigh draw,
 * words 1 and 2 the Gaussian one.  d_counters [n][4] and d_out [n][4] uint32,
 * device, 16-byte aligned; d_out may equal d_counters.  Errors: SONAR_ERR_ARG
 * (n < 0, NULL or unaligned buffers with n > 0), before anything is enqueued. */
sonar_status sonar_philox(sonar_ctx_t ctx, const uint32_t* d_counters, int64_t n, uint64_t seed, uint32_t* d_out,
                          void* stream);

/* L2 read bandwidth: reads the caller's buffer `passes` times over with
 * 16-byte loads that are cached in L2 but not in L1, on n_blocks blocks of
 * 512 threads, and writes each block's sum of the values it read (FP32) to
 * d_block_sums[n_blocks].  A buffer well below the L2 size (e.g. 32 MiB)
 * stays resident after the first pass, so bytes * passes / duration measures
 * the L2 read rate that the ray cast's node and triangle fetches draw on.
 * d_buf 16-byte aligned device memory of `bytes` (a multiple of 16, > 0);
 * passes >= 1; 1 <= n_blocks <= 65535.  Errors: SONAR_ERR_ARG, before
 * anything is enqueued. */
sonar_status sonar_probe_l2_read(sonar_ctx_t ctx, const void* d_buf, int64_t bytes, int32_t passes,
                                 float* d_block_sums, int32_t n_blocks, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SONAR_H */
