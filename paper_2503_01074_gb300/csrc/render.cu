// Sonar post-processing kernels (OceanSim, arXiv 2503.01074, Sec. III-A-2).
//
// k_bin               one work unit = whole azimuth columns of one sensor: the
//                     units' hit records -> intensity (Eq. 2, two-way) -> polar
//                     binning into a shared-memory column block -> Eq. 3-6 noise
//                     per bin -> I~ to HBM.  A unit owns its columns, so every
//                     polar bin is written exactly once: no global atomics, no
//                     memset of the image.
// k_norm_rows         range-wise normalisation: one warp per range row takes the
//                     row maximum of I~ and writes N = I~ / max.
// k_fan_*             fan resample of the normalised image: per-pixel polar
//                     coordinate tables, then bilinear gathers for up to 8
//                     frames per table read.
// adjoint             per-group (row) Jacobian terms, then a per-ray gather of
//                     dL/dP into (dalpha, dgain, dmu) over ray chunks, and a
//                     fixed-order final reduction (deterministic).
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "sonar_host.h"
#include "sonar_internal.cuh"
#include "devmath.cuh"

namespace sonar {
namespace {

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
// The additive term of Eq. 3 for range row `row` (centre r_c) and a column
// whose beam-pattern factor 0.5 exp(-phi_c^2 / sigma_phi) is `pat`, from the
// bin's uniform word of the additive stream: (r_c^2 / r_max^2)(1 + pat w_sa),
// w_sa ~ Rayleigh(sigma_sa) (Eq. 4).
struct AdditiveTerm {
    float dr, rmin, inv_rmax2, sig_sa;
    __device__ __forceinline__ float operator()(int row, float pat, uint32_t word) const {
        const float w_sa = rayleigh_of(word, sig_sa);
        const float rc = fmaf(small_u2f(row) + 0.5f, dr, rmin);
        return rc * rc * inv_rmax2 * (1.0f + pat * w_sa);
    }
};

template <int DET>
__global__ void __launch_bounds__(512) k_bin(BinArgs a) {
    extern __shared__ __align__(16) float acc[];
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
    int clean_nbin = -1;   // block-uniform: the unit size whose accumulator and bitmap are known zero
    int next_u = 0;   // thread 0: the unit taken ahead, while the block works on the current one
    for (int iter = 0;; ++iter) {
        int u;
        if (a.work_counter) {
            if (tid == 0) s_unit = iter == 0 ? atomicAdd(a.work_counter, 1) : next_u;
            __syncthreads();
            u = s_unit;
            if (tid == 0 && u < a.n_units) next_u = atomicAdd(a.work_counter, 1);
        } else {
            if (iter > 0) break;
            u = blockIdx.x;
        }
        if (u >= a.n_units) break;
        if (a.units) {   // warp 0 fetches the unit, then its sensor and scene descriptors at once
            if (warp == 0) {
                const Unit un = a.units[u];
                copy_words(&S, a.sensors + un.sensor, lane);
                copy_words(&SC, a.scenes + un.scene, lane);
                if (lane == 0) U = un;
            }
        } else if (tid == 0) {
            load_unit(a, u, &S, &SC, &U);
        }
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
        // the list of bins with returns holds one entry per ray at most (only a
        // bin that a ray lands in can be nonzero): the host sizes it so
        const int lcap = (int)min((int64_t)nbin, r1 - r0);
        // Noise first: with at most one beam per column and no whole-image
        // maximum, a bin's additive term does not depend on the fold, so pass 1
        // writes it for every bin before the rays are folded (the fold's record
        // loads then meet a busy block rather than a barrier); the fold lists each
        // bin at its first return (a shared bitmap), and pass 2 finishes and
        // resets only the listed bins, which leaves the accumulator and bitmap
        // zero for the next unit of the same size.
        if (DET && !per_beam && S.nb <= S.naz && a.params.normalise != 2) {
            uint32_t* bits = reinterpret_cast<uint32_t*>(acc + nbin);
            const int nwords = (nbin + 31) >> 5;
            int* flist = reinterpret_cast<int*>(bits + nwords);
            if (clean_nbin != nbin)
                for (int k = tid; k < nbin + nwords; k += nt) acc[k] = 0.0f;   // bitmap words too (0.0f is 0)
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
            const PhiloxKey K = philox_key(S.seed_lo, S.seed_hi);
            const uint32_t naz_r = (uint32_t)S.naz, c0_r = (uint32_t)U.c0, flo = S.frame_lo, fhi = S.frame_hi;
            const float rmin_r = S.rmin;
            const AdditiveTerm additive{dr, rmin_r, inv_rmax2, sig_sa};
            float* const noised_r = a.noised + S.polar_off;
            float* const binned_r = a.binned ? a.binned + S.polar_off : nullptr;
            if (((naz_r | c0_r | (uint32_t)cw) & 3u) == 0) {
                const int cq = cw >> 2, nquad = S.nr * cq;
                const int dqr = nt / cq, dqc = nt - dqr * cq;
                int row = tid / cq, qc = tid - row * cq;
                const bool vec = ((reinterpret_cast<uintptr_t>(noised_r) |
                                   reinterpret_cast<uintptr_t>(binned_r)) & 15u) == 0;
                for (int g = tid; g < nquad; g += nt) {
                    const uint32_t b0 = (uint32_t)row * naz_r + c0_r + 4u * (uint32_t)qc;
                    const U4 x = additive_words(b0 >> 2, flo, fhi, K);
                    const uint32_t xw[4] = {x.x, x.y, x.z, x.w};
                    float add[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) add[j] = additive(row, s_pat[4 * qc + j], xw[j]);
                    if (vec) {
                        *reinterpret_cast<float4*>(noised_r + b0) = make_float4(add[0], add[1], add[2], add[3]);
                        if (binned_r) *reinterpret_cast<float4*>(binned_r + b0) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            noised_r[b0 + j] = add[j];
                            if (binned_r) binned_r[b0 + j] = 0.0f;
                        }
                    }
                    row += dqr;
                    qc += dqc;
                    if (qc >= cq) { qc -= cq; ++row; }
                }
            } else {
                const int drow = nt / cw, dcol = nt - drow * cw;
                int row = tid / cw, col = tid - row * cw;
                for (int k = tid; k < nbin; k += nt) {
                    const uint32_t b = (uint32_t)row * naz_r + c0_r + (uint32_t)col;
                    const U4 x = additive_words(b >> 2, flo, fhi, K);
                    noised_r[b] = additive(row, s_pat[col], word_of(x, b & 3u));
                    if (binned_r) binned_r[b] = 0.0f;
                    row += drow;
                    col += dcol;
                    if (col >= cw) { col -= cw; ++row; }
                }
            }
            // the fold: warp w takes beams w, w + nw, ... of the unit, each in
            // elevation order (its column's canonical order)
            for (int bb = warp; bb < nbeam; bb += nw) {
                const sonar_hit* Hb = H + (int64_t)(i0 + bb) * S.ne;
                for (int jb = 0; jb < S.ne; jb += 32) {
                    const int j = jb + lane;
                    uint32_t lkey = kNoKey;
                    float score = 0.0f;
                    if (j < S.ne) {
                        const uint4 h = __ldg(reinterpret_cast<const uint4*>(Hb + j));
                        if (h.x != kNoKey) {
                            const uint32_t br = h.x / naz_r, ba = h.x - br * naz_r;
                            lkey = br * (uint32_t)cw + (ba - c0_r);
                            if (lkey >= (uint32_t)nbin || h.y >= (uint32_t)SC.n_tris) {   // not this unit's bin: a corrupt record
                                atomicOr(a.err, SONAR_DEVERR_INDEX);
                                lkey = kNoKey;
                            }
                            int m = lkey == kNoKey ? 0 : SC.mat_orig[h.y];
                            m = m < a.n_mat ? m : a.n_mat - 1;
                            score = __ldg(a.theta + 2 + m) * __uint_as_float(h.w) *
                                    expf(-2.0f * alpha * __uint_as_float(h.z)) * gain;
                        }
                    }
                    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, lkey);
                    if (lkey != kNoKey) {
                        const int leader = __ffs(peers) - 1;
                        float v = lane == leader ? acc[lkey] : 0.0f;
                        for (uint32_t m = peers; m; m &= m - 1) v += __shfl_sync(peers, score, __ffs(m) - 1);
                        if (lane == leader) {
                            acc[lkey] = v;
                            const uint32_t bit = 1u << (lkey & 31u);
                            if (!(atomicOr(&bits[lkey >> 5], bit) & bit)) {
                                const int q = atomicAdd(&s_count, 1);
                                if (q < lcap) flist[q] = (int)lkey;
                                else atomicOr(a.err, SONAR_DEVERR_INDEX);
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // pass 2: the listed bins get P (0.5 + w_sm) on top of the additive
            // term written by pass 1 (visible after the barrier), then are reset
            const int nl = min(s_count, lcap);
            for (int q = tid; q < nl; q += nt) {
                const int k = flist[q];
                const int rw = k / cw, cl = k - rw * cw;
                const uint32_t b = (uint32_t)rw * naz_r + c0_r + (uint32_t)cl;
                const float P = acc[k];
                acc[k] = 0.0f;
                bits[k >> 5] = 0u;
                if (binned_r) binned_r[b] = P;
                if (P != 0.0f) {
                    const float w_sm = gauss_of(bin_draws(b, S, K), sig_sm);
                    noised_r[b] = P * (0.5f + w_sm) + noised_r[b];
                }
            }
            clean_nbin = nbin;
            __syncthreads();
            continue;
        }
        clean_nbin = -1;   // the path below leaves its accumulator in use
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
        // With at most one beam per column (n_beams <= n_az_bins) a beam's bins
        // are its column's own: warp w folds beams w, w + nw, ... straight into
        // the unit's accumulator, each in elevation order (the canonical order of
        // that column's rays, so the same sums as the turn-taking fold below),
        // with no barriers between warps.
        const bool col_fold = DET && !per_beam && S.nb <= S.naz;
        if (col_fold) {
            const uint32_t naz = (uint32_t)S.naz;
            for (int bb = warp; bb < nbeam; bb += nw) {
                const sonar_hit* Hb = H + (int64_t)(i0 + bb) * S.ne;
                for (int jb = 0; jb < S.ne; jb += 32) {
                    const int j = jb + lane;
                    uint32_t lkey = kNoKey;
                    float score = 0.0f;
                    if (j < S.ne) {
                        const uint4 h = __ldg(reinterpret_cast<const uint4*>(Hb + j));
                        if (h.x != kNoKey) {
                            const uint32_t br = h.x / naz, ba = h.x - br * naz;
                            lkey = br * (uint32_t)cw + (ba - (uint32_t)U.c0);
                            int m = SC.mat_orig[h.y];
                            m = m < a.n_mat ? m : a.n_mat - 1;
                            score = __ldg(a.theta + 2 + m) * __uint_as_float(h.w) *
                                    expf(-2.0f * alpha * __uint_as_float(h.z)) * gain;
                        }
                    }
                    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, lkey);
                    if (lkey != kNoKey) {
                        const int leader = __ffs(peers) - 1;
                        float v = lane == leader ? acc[lkey] : 0.0f;
                        for (uint32_t m = peers; m; m &= m - 1) v += __shfl_sync(peers, score, __ffs(m) - 1);
                        if (lane == leader) acc[lkey] = v;
                    }
                }
            }
        }
        for (int64_t base = r0; base < (per_beam || col_fold ? r0 : r1); base += nt) {
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
        // Eq. 3-6 per bin.  Pass 1 visits every bin: the additive Rayleigh term,
        // which is already the final value of a bin without returns (P = 0 makes
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
        const PhiloxKey K = philox_key(S.seed_lo, S.seed_hi);
        // the sensor fields this loop reads, in registers (the loop's shared-memory
        // stores would otherwise make the compiler reload them every bin)
        const uint32_t naz_r = (uint32_t)S.naz, c0_r = (uint32_t)U.c0, flo = S.frame_lo, fhi = S.frame_hi;
        const float rmin_r = S.rmin;
        const AdditiveTerm additive{dr, rmin_r, inv_rmax2, sig_sa};
        float* const noised_r = a.noised + S.polar_off;
        float* const binned_r = a.binned ? a.binned + S.polar_off : nullptr;
        // Pass 1 writes every bin's additive term to I~ (pass 2 adds the
        // multiplicative term of the listed bins to it).  When the unit's bins
        // come in aligned fours (row width, first column and unit width multiples
        // of 4) a thread takes four neighbouring bins: one Philox block gives
        // their four additive draws, and they move as 16-byte vectors.
        if (((naz_r | c0_r | (uint32_t)cw) & 3u) == 0) {
            const int cq = cw >> 2, nquad = S.nr * cq;
            const int dqr = nt / cq, dqc = nt - dqr * cq;
            int row = tid / cq, qc = tid - row * cq;
            const bool vec = ((reinterpret_cast<uintptr_t>(noised_r) |
                               reinterpret_cast<uintptr_t>(binned_r)) & 15u) == 0;
            for (int g = tid; g < nquad; g += nt) {
                const int k0 = row * cw + 4 * qc;
                const uint32_t b0 = (uint32_t)row * naz_r + c0_r + 4u * (uint32_t)qc;
                float P[4];
                if (per_beam) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        P[j] = 0.0f;
                        for (int bb = s_b0[4 * qc + j]; bb < s_b0[4 * qc + j + 1]; ++bb) P[j] += accb[bb * S.nr + row];
                    }
                } else {
                    const float4 v = *reinterpret_cast<const float4*>(acc + k0);
                    P[0] = v.x; P[1] = v.y; P[2] = v.z; P[3] = v.w;
                }
                const U4 x = additive_words(b0 >> 2, flo, fhi, K);
                const uint32_t xw[4] = {x.x, x.y, x.z, x.w};
                float add[4], keep[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    add[j] = additive(row, s_pat[4 * qc + j], xw[j]);
                    keep[j] = add[j];
                    if (P[j] != 0.0f) {
                        keep[j] = P[j];
                        const int q = atomicAdd(&s_count, 1);
                        if (q < lcap) list[q] = k0 + j;
                        else atomicOr(a.err, SONAR_DEVERR_INDEX);
                    }
                }
                if (vec) {
                    *reinterpret_cast<float4*>(noised_r + b0) = make_float4(add[0], add[1], add[2], add[3]);
                    if (binned_r) *reinterpret_cast<float4*>(binned_r + b0) = make_float4(P[0], P[1], P[2], P[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        noised_r[b0 + j] = add[j];
                        if (binned_r) binned_r[b0 + j] = P[j];
                    }
                }
                *reinterpret_cast<float4*>(acc + k0) = make_float4(keep[0], keep[1], keep[2], keep[3]);
                row += dqr;
                qc += dqc;
                if (qc >= cq) { qc -= cq; ++row; }
            }
        } else {
            const int drow = nt / cw, dcol = nt - drow * cw;
            int row = tid / cw, col = tid - row * cw;
            for (int k = tid; k < nbin; k += nt) {
                const uint32_t b = (uint32_t)row * naz_r + c0_r + (uint32_t)col;
                float P;
                if (per_beam) {
                    P = 0.0f;
                    for (int bb = s_b0[col]; bb < s_b0[col + 1]; ++bb) P += accb[bb * S.nr + row];
                } else {
                    P = acc[k];
                }
                const U4 x = additive_words(b >> 2, flo, fhi, K);
                const float add = additive(row, s_pat[col], word_of(x, b & 3u));
                if (binned_r) binned_r[b] = P;
                noised_r[b] = add;
                if (P != 0.0f) {
                    acc[k] = P;
                    const int q = atomicAdd(&s_count, 1);
                    if (q < lcap) list[q] = k;
                    else atomicOr(a.err, SONAR_DEVERR_INDEX);
                } else {
                    acc[k] = add;
                }
                row += drow;
                col += dcol;
                if (col >= cw) { col -= cw; ++row; }
            }
        }
        __syncthreads();
        // Pass 2: the listed bins (P != 0) add P (0.5 + w_sm) to the additive
        // term that pass 1 wrote (visible to the block after the barrier)
        const int nlist = min(s_count, lcap);
        for (int q = tid; q < nlist; q += nt) {
            const int k = list[q];
            const int rw = k / cw, cl = k - rw * cw;
            const uint32_t b = (uint32_t)(rw * S.naz + U.c0 + cl);
            const float P = acc[k];
            const float w_sm = gauss_of(bin_draws(b, S, K), sig_sm);
            const float In = P * (0.5f + w_sm) + noised_r[b];
            noised_r[b] = In;
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

// The noise stream itself: Philox4x32-10 of n counters under one key, the
// same round function the binning, adjoint and DVL kernels draw from.
__global__ void __launch_bounds__(256) k_philox_words(const uint4* ctr, int64_t n, uint32_t k0, uint32_t k1,
                                                      uint4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    const U4 x = philox10(U4{c.x, c.y, c.z, c.w}, philox_key(k0, k1));
    out[i] = make_uint4(x.x, x.y, x.z, x.w);
}

__device__ __forceinline__ float norm_value(float In, float m, int mode) {
    return (mode != 0 && m > 0.0f) ? In / m : In;
}

// One row: its maximum over azimuth and N = I~ / max (any alignment and width).
__device__ __forceinline__ void norm_row(const NormArgs& a, int64_t g, int lane) {
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

// One warp per pair of adjacent range rows, the pairs from the last to the
// first: the binning kernel wrote the last sensors' I~ last, so the first rows
// read here are still in L2, and the first sensors' N, written last, are in L2
// when the fan starts on them.  A row of 16-byte-aligned bins, at most 512 of
// them, stays in registers between its maximum and the division, and both rows'
// loads are issued before either reduction (4 KB in flight per warp); other
// rows go one at a time (in registers up to 1024 aligned bins, else in two
// passes).
__global__ void __launch_bounds__(256, 4) k_norm_rows(NormArgs a) {
    constexpr int kV = 4;   // float4 per lane: rows of up to 512 bins
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t pairs = (a.total_rows + 1) >> 1;
    if (t >= pairs) return;
    const int64_t g0 = 2 * (pairs - 1 - t);
    float4 v[2][kV];
    float4* out4[2] = {nullptr, nullptr};
    int n4[2] = {0, 0};
    bool fast[2] = {false, false};
    int64_t rowmax_off[2] = {0, 0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t g = g0 + r;
        if (g >= a.total_rows) continue;
        const SensorDev& s = a.sensors ? a.sensors[a.row_map[g]] : a.one;
        const int naz = s.naz;
        if (((s.polar_off | naz) & 3) != 0 || naz > 32 * 4 * kV) continue;
        const int64_t off = s.polar_off + (int64_t)(g - s.rowmax_off) * naz;
        const float4* In4 = reinterpret_cast<const float4*>(a.noised + off);
        out4[r] = reinterpret_cast<float4*>(a.polar + off);
        n4[r] = naz >> 2;
        fast[r] = true;
        rowmax_off[r] = s.rowmax_off;
#pragma unroll
        for (int k = 0; k < kV; ++k) {
            const int q = lane + 32 * k;
            v[r][k] = q < n4[r] ? __ldg(In4 + q)
                                : make_float4(-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F);
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t g = g0 + r;
        if (g >= a.total_rows) continue;
        if (!fast[r]) {
            norm_row(a, g, lane);
            continue;
        }
        float m = 0.0f;
        if (a.normalise == 1) {
            m = -CUDART_INF_F;
#pragma unroll
            for (int k = 0; k < kV; ++k) m = fmaxf(fmaxf(m, fmaxf(v[r][k].x, v[r][k].y)), fmaxf(v[r][k].z, v[r][k].w));
            for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        } else if (a.normalise == 2) {
            m = ord_dec(a.gmax[rowmax_off[r]]);
        }
#pragma unroll
        for (int k = 0; k < kV; ++k) {
            const int q = lane + 32 * k;
            if (q < n4[r])
                out4[r][q] = make_float4(norm_value(v[r][k].x, m, a.normalise), norm_value(v[r][k].y, m, a.normalise),
                                         norm_value(v[r][k].z, m, a.normalise), norm_value(v[r][k].w, m, a.normalise));
        }
    }
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

// One block = a kTileSide x kTileSide square of one sensor's fan (a square
// maps to a compact patch of the polar image, so its gathers stay in cache);
// lane x of a kTileSide-thread row takes column x, rows step by 256 / kTileSide.
// A sensor with a coordinate table reads its pixels' coordinates from it.
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
    const int sx = (S.fan_w + kTileSide - 1) / kTileSide;
    const int u = (s_sq % sx) * kTileSide + (threadIdx.x & (kTileSide - 1));
    const int v0 = (s_sq / sx) * kTileSide + (threadIdx.x / kTileSide);
    if (u >= S.fan_w) return;
    const float* P = a.polar + S.polar_off;
    float* F = a.fan + S.fan_off;
    const uint4* lut = S.fan_lut;
#pragma unroll 4
    for (int k = 0; k < kTileSide; k += 256 / kTileSide) {
        const int v = v0 + k;
        if (v >= S.fan_h) break;
        const int64_t pix = (int64_t)v * S.fan_w + u;
        __stcs(F + pix, fan_blend(lut ? __ldg(lut + pix) : fan_coord(S, pix), P));   // never re-read here: stream past L2
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
                // the fan is never re-read by the step: streaming stores leave L2
                // to the polar images and the coordinate table
                __stcs(a.fan + M[q].fan_off + pix, fan_blend(cq, a.polar + M[q].polar_off));
            }
        }
    }
}

// Fills the coordinate table of each owner sensor (one block = kFanTile
// pixels).  A block whose stamp already holds the owner's fan_version has
// nothing to do: the table depends on the fan geometry only, and the host bumps
// the version whenever an update changes it.
__global__ void __launch_bounds__(256) k_fan_lut(FanLutArgs a) {
    __shared__ SensorDev S;
    __shared__ int s_blk;
    __shared__ uint4* s_lut;
    if (threadIdx.x == 0) {
        const int2 m = a.block_map[blockIdx.x];
        S = a.sensors[m.x];
        s_blk = m.y;
        s_lut = a.luts[m.x];
    }
    __syncthreads();
    if (S.fan_stamp && S.fan_stamp[s_blk] == S.fan_version) return;   // block-uniform
    const int64_t base = (int64_t)s_blk * kFanTile;
    const int64_t n = (int64_t)S.fan_w * S.fan_h;
#pragma unroll 1
    for (int k = 0; k < kFanTile / 256; ++k) {
        const int64_t pix = base + k * 256 + threadIdx.x;
        if (pix < n) s_lut[pix] = fan_coord(S, pix);
    }
    // the entries are read by later launches only, which see both them and the stamp
    if (threadIdx.x == 0 && S.fan_stamp) S.fan_stamp[s_blk] = S.fan_version;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------

// Group terms of the normalisation Jacobian: m, argmax (lowest index on
// ties) and c = sum G I~ / m^2.  Mode 1: one warp per range row; mode 2: one
// block per sensor image.
__global__ void k_adj_rows(const SensorDev* sensors, const int32_t* row_map, SensorDev one, int n_sensors,
                           int64_t total, int mode, const float* noised, const float* grad, RowInfo* info,
                           int32_t* zero_word) {
    const int lane = threadIdx.x & 31;
    if (zero_word && blockIdx.x == 0 && threadIdx.x == 0) *zero_word = 0;   // the gather's work counter
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
        if (((s.polar_off | s.naz) & 3) == 0 && s.naz <= 512) {
            // 16-byte rows of up to 512 bins: every load of the row (I~ and G) is
            // issued before the first compare, then each lane takes its 4
            // consecutive bins per vector in index order
            const float4* In4 = reinterpret_cast<const float4*>(In);
            const float4* G4 = reinterpret_cast<const float4*>(G);
            const int n4 = s.naz >> 2;
            float4 xs[4], ys[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = lane + 32 * k;
                if (q < n4) {
                    xs[k] = __ldcs(In4 + q);   // I~ is not read again by the adjoint: evict first, keep G in L2
                    ys[k] = __ldg(G4 + q);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = lane + 32 * k;
                if (q >= n4) continue;
                const float4 x = xs[k], y = ys[k];
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
        } else if (((s.polar_off | s.naz) & 3) == 0) {
            // wider 16-byte rows: each lane takes 4 consecutive bins per load, in index order
            const float4* In4 = reinterpret_cast<const float4*>(In);
            const float4* G4 = reinterpret_cast<const float4*>(G);
#pragma unroll 4
            for (int q = lane; q < (s.naz >> 2); q += 32) {
                const float4 x = __ldcs(In4 + q), y = __ldg(G4 + q);
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
    int next_u = 0;   // thread 0: the unit taken ahead
    for (int iter = 0;; ++iter) {
        int u;
        if (a.work_counter) {
            if (tid == 0) s_unit = iter == 0 ? atomicAdd(a.work_counter, 1) : next_u;
            __syncthreads();
            u = s_unit;
            if (tid == 0 && u < a.n_units) next_u = atomicAdd(a.work_counter, 1);
        } else {
            if (iter > 0) break;
            u = blockIdx.x;
        }
        if (u >= a.n_units) break;
        if (a.units && warp == 0) {   // warp 0 fetches the unit, then its sensor and scene descriptors at once
            const AdjUnit un = a.units[u];
            copy_words(&S, a.sensors + un.sensor, lane);
            copy_words(&SC, a.scenes + un.scene, lane);
            if (lane == 0) U = un;
        }
        if (!a.units && tid == 0) {
            S = a.one;
            SC = a.one_scene;
            U.sensor = 0;
            U.r0 = u * a.chunk;
            U.r1 = min(U.r0 + a.chunk, a.one.nb * a.one.ne);
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
            // material sums of this warp: one butterfly reduction (a fixed order,
            // so deterministic) per distinct material among the valid lanes,
            // added to the slab by the material's lowest lane
            uint32_t todo = __ballot_sync(0xFFFFFFFFu, valid);
            while (todo) {
                const int leader = __ffs(todo) - 1;
                const int m = __shfl_sync(0xFFFFFFFFu, mat, leader);
                const bool mine = valid && mat == m;
                float x = mine ? v_mu : 0.0f;
                for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
                if (lane == leader) slab[warp * nm + m] += x;
                todo &= ~__ballot_sync(0xFFFFFFFFu, mine);
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
}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

void set_kernel_attributes() {
    cudaFuncSetAttribute(k_bin<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    cudaFuncSetAttribute(k_bin<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
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

cudaError_t launch_philox(const void* ctr, int64_t n, uint32_t k0, uint32_t k1, void* out, cudaStream_t st) {
    if (n > 0)
        k_philox_words<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(static_cast<const uint4*>(ctr), n, k0, k1,
                                                                      static_cast<uint4*>(out));
    return cudaGetLastError();
}

cudaError_t launch_norm(const NormArgs& a, cudaStream_t st) {
    const int64_t threads = ((a.total_rows + 1) / 2) * 32;   // a warp per pair of rows
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
                            const float* grad, RowInfo* info, int32_t* zero_word, cudaStream_t st) {
    if (normalise == 1) {
        const int64_t threads = total_groups * 32;
        k_adj_rows<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(sensors, row_map, one, n_sensors,
                                                                      total_groups, 1, noised, grad, info,
                                                                      zero_word);
    } else if (normalise == 2) {
        k_adj_rows<<<(unsigned)total_groups, 1024, 0, st>>>(sensors, row_map, one, n_sensors, total_groups, 2,
                                                            noised, grad, info, zero_word);
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

}  // namespace sonar
