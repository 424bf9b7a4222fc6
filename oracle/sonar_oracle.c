/*
 * sonar_oracle.c -- plain FP64 CPU oracle for forward-looking imaging-sonar
 * rendering (OceanSim, arXiv 2503.01074, Sec. III-A-2, Eq. 2-6).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the package smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Every step is the plain definition, in the order the method applies it:
 *   rays        one ray per (beam i, elevation j) cell centre of the field of view
 *   closest hit brute force over every triangle, Moller-Trumbore in FP64
 *   intensity   s = mu[m] * cos * exp(-2 alpha r) * gain          (Eq. 2, two-way)
 *   binning     sum of s over the returns in each (range, azimuth) cell (Sec. III-A-2)
 *   noise       I~ = I (0.5 + w_sm) + r^2/r_max^2 (1 + 0.5 exp(-phi^2/sigma_phi) w_sa)
 *               w_sa ~ Rayleigh(sigma_sa), w_sm ~ N(0, sigma_sm)      (Eq. 3-6)
 *   normalise   range-wise: each range row divided by its maximum (Sec. III-A-2)
 *   fan         Cartesian resample of the polar image (plot style, Sec. III-A-2)
 *   gradient    analytic adjoint of the above w.r.t. (alpha, gain, mu)
 *   camera      underwater image formation of an in-air image and its depth (Eq. 1)
 *   DVL         four-beam Janus ranges, least-squares velocity, rate and dropout
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11), written from that paper's description.
 *
 * Sensor descriptor (double[20]):
 *   [0..2] position, [3..11] sensor->world rotation (row-major),
 *   [12] n_beams, [13] n_elev, [14] n_range_bins, [15] n_az_bins,
 *   [16] hfov (rad), [17] vfov (rad), [18] r_min (m), [19] r_max (m).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define SD_NB 12
#define SD_NE 13
#define SD_NR 14
#define SD_NAZ 15
#define SD_HFOV 16
#define SD_VFOV 17
#define SD_RMIN 18
#define SD_RMAX 19

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

/* One Philox-4x32 round: two 32x32->64 multiplications of words 0 and 2 by
 * the round multipliers; the high halves are xored with the other two words
 * and the round key, the low halves pass through, with the words permuted. */
static void philox_round(uint32_t x[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x[1] ^ k[0];
    const uint32_t y1 = (uint32_t)p1;
    const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x[3] ^ k[1];
    const uint32_t y3 = (uint32_t)p0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

/* Ten rounds; the key is bumped by the Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(x, k);
    }
    memcpy(out, x, sizeof x);
}

void oracle_philox_batch(const uint32_t* ctr, int64_t n, const uint32_t key[2], uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* uniform on (0, 1]: (x + 1) / 2^32, exact in FP64 */
static double u01(uint32_t x) { return ((double)x + 1.0) * 0x1p-32; }

/* The per-bin draws of Eq. 4 and 5, key = seed.  Additive term: Rayleigh(sigma_sa)
 * by inversion of word (bin mod 4) of counter (bin / 4, frame lo, 1, frame hi),
 * so four neighbouring bins share one block of the stream.  Multiplicative term:
 * N(0, sigma_sm) by the Box-Muller cosine branch of words 1, 2 of counter (bin,
 * frame lo, 0, frame hi); its words 0 and 3 are unused.  Counter word 2 tells
 * the two streams apart. */
static void bin_draws(uint64_t bin, uint64_t seed, uint64_t frame, double sigma_sa,
                      double sigma_sm, double* w_sa, double* w_sm)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ca[4] = {(uint32_t)(bin >> 2), (uint32_t)frame, 1u, (uint32_t)(frame >> 32)};
    const uint32_t cm[4] = {(uint32_t)bin, (uint32_t)frame, 0u, (uint32_t)(frame >> 32)};
    uint32_t xa[4], xm[4];
    oracle_philox4x32_10(ca, key, xa);
    oracle_philox4x32_10(cm, key, xm);
    *w_sa = sigma_sa * sqrt(-2.0 * log(u01(xa[bin & 3u])));
    *w_sm = sigma_sm * sqrt(-2.0 * log(u01(xm[1]))) * cos(2.0 * M_PI * u01(xm[2]));
}

void oracle_noise_draws(int64_t n_bins, uint64_t seed, uint64_t frame, double sigma_sa,
                        double sigma_sm, double* w_sa, double* w_sm)
{
    for (int64_t b = 0; b < n_bins; ++b)
        bin_draws((uint64_t)b, seed, frame, sigma_sa, sigma_sm, w_sa + b, w_sm + b);
}

/* ------------------------------------------------------------------------ */
/* Rays                                                                      */
/* ------------------------------------------------------------------------ */

/* Beam i at azimuth phi_i = -H/2 + (i + 1/2) H / N_b, elevation j at
 * theta_j = -V/2 + (j + 1/2) V / N_e; sensor-frame direction
 * (sin phi cos theta, cos phi cos theta, sin theta), rotated to the world and
 * normalised.  Ray k = i * N_e + j. */
void oracle_ray_dirs(const double* sd, double* dirs)
{
    const int nb = (int)sd[SD_NB], ne = (int)sd[SD_NE];
    const double H = sd[SD_HFOV], V = sd[SD_VFOV];
    const double* R = sd + 3;
    for (int i = 0; i < nb; ++i) {
        const double phi = -H / 2.0 + (i + 0.5) * H / nb;
        for (int j = 0; j < ne; ++j) {
            const double th = -V / 2.0 + (j + 0.5) * V / ne;
            const double ds[3] = {sin(phi) * cos(th), cos(phi) * cos(th), sin(th)};
            double dw[3];
            for (int a = 0; a < 3; ++a)
                dw[a] = R[3 * a + 0] * ds[0] + R[3 * a + 1] * ds[1] + R[3 * a + 2] * ds[2];
            const double n = sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
            double* d = dirs + 3 * ((int64_t)i * ne + j);
            d[0] = dw[0] / n; d[1] = dw[1] / n; d[2] = dw[2] / n;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Closest hit: brute force over all triangles                               */
/* ------------------------------------------------------------------------ */

/* Moller-Trumbore: hit iff det != 0, u >= 0, v >= 0, u + v <= 1, t > 0. */
static int moller_trumbore(const double o[3], const double d[3], const float* tv,
                           double* t, double* u, double* v)
{
    const double v0[3] = {tv[0], tv[1], tv[2]};
    const double e1[3] = {tv[3] - v0[0], tv[4] - v0[1], tv[5] - v0[2]};
    const double e2[3] = {tv[6] - v0[0], tv[7] - v0[1], tv[8] - v0[2]};
    const double p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2],
                         d[0] * e2[1] - d[1] * e2[0]};
    const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    if (det == 0.0) return 0;
    const double inv = 1.0 / det;
    const double s[3] = {o[0] - v0[0], o[1] - v0[1], o[2] - v0[2]};
    const double uu = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
    if (uu < 0.0 || uu > 1.0) return 0;
    const double q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2],
                         s[0] * e1[1] - s[1] * e1[0]};
    const double vv = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
    if (vv < 0.0 || uu + vv > 1.0) return 0;
    const double tt = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
    if (!(tt > 0.0)) return 0;
    *t = tt; *u = uu; *v = vv;
    return 1;
}

typedef struct {
    const float* tv;      /* [nt][9] triangle vertices (v0, v1, v2), FP32 input */
    int64_t nt;
    const double* o;      /* [3] */
    const double* dirs;   /* [nr][3] */
    int64_t nr;
    double t_max;
    int32_t* tri; double* t; double* u; double* v; double* t2; double* dn;
    int nthreads, tid;
} trace_job;

static void trace_one(const trace_job* J, int64_t k)
{
    const double* d = J->dirs + 3 * k;
    int64_t best = -1;
    double bt = INFINITY, bu = 0, bv = 0, t2 = INFINITY;
    for (int64_t f = 0; f < J->nt; ++f) {
        double t, u, v;
        if (!moller_trumbore(J->o, d, J->tv + 9 * f, &t, &u, &v)) continue;
        if (!(t < J->t_max)) continue;
        if (t < bt || (t == bt && f < best)) {
            if (best >= 0) t2 = bt;           /* the displaced nearest becomes second */
            best = f; bt = t; bu = u; bv = v;
        } else if (t < t2) {
            t2 = t;
        }
    }
    J->tri[k] = (int32_t)best;
    J->t[k] = best >= 0 ? bt : INFINITY;
    J->u[k] = bu; J->v[k] = bv; J->t2[k] = t2;
    if (best >= 0) {
        const float* tv = J->tv + 9 * best;
        const double e1[3] = {(double)tv[3] - tv[0], (double)tv[4] - tv[1], (double)tv[5] - tv[2]};
        const double e2[3] = {(double)tv[6] - tv[0], (double)tv[7] - tv[1], (double)tv[8] - tv[2]};
        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        J->dn[k] = (d[0] * n[0] + d[1] * n[1] + d[2] * n[2]) / nn;
    } else {
        J->dn[k] = 0.0;
    }
}

static void* trace_worker(void* arg)
{
    const trace_job* J = (const trace_job*)arg;
    for (int64_t k = J->tid; k < J->nr; k += J->nthreads) trace_one(J, k);
    return NULL;
}

/* For each ray: nearest triangle (-1 = miss), its t, barycentrics (u, v),
 * the nearest t on any other triangle (t2), and d . n_hat with the geometric
 * normal n = (v1 - v0) x (v2 - v0).  Hits need t < t_max (INFINITY = none).
 * Exact ties in t go to the lower triangle index. */
int oracle_closest_hits(const float* tri_verts, int64_t nt, const double* origin,
                        const double* dirs, int64_t nr, double t_max, int nthreads,
                        int32_t* tri, double* t, double* u, double* v, double* t2, double* dn)
{
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    trace_job jobs[256];
    for (int w = 0; w < nthreads; ++w) {
        jobs[w] = (trace_job){tri_verts, nt, origin, dirs, nr, t_max, tri, t, u, v, t2, dn,
                              nthreads, w};
        if (pthread_create(&th[w], NULL, trace_worker, &jobs[w]) != 0) {
            trace_worker(&jobs[w]);
            th[w] = 0;
        }
    }
    for (int w = 0; w < nthreads; ++w)
        if (th[w]) pthread_join(th[w], NULL);
    return nthreads;
}

/* ------------------------------------------------------------------------ */
/* Intensity and binning                                                     */
/* ------------------------------------------------------------------------ */

/* The incidence factor: |d . n| for two-sided surfaces, else max(0, -d . n). */
static double incidence(double dn, int two_sided)
{
    if (two_sided) return fabs(dn);
    return -dn > 0.0 ? -dn : 0.0;
}

/* Eq. 2 in its two-way form: s = mu[m] * cos * exp(-2 alpha r) * gain. */
void oracle_scores(int64_t nr, const int32_t* tri, const double* t, const double* dn,
                   const int32_t* mat_of_tri, const double* mu, double alpha, double gain,
                   int two_sided, double* s)
{
    for (int64_t k = 0; k < nr; ++k) {
        if (tri[k] < 0) { s[k] = 0.0; continue; }
        s[k] = mu[mat_of_tri[tri[k]]] * incidence(dn[k], two_sided) * exp(-2.0 * alpha * t[k]) * gain;
    }
}

/* Range bin floor((r - r_min) N_r / (r_max - r_min)) for r_min <= r < r_max;
 * azimuth bin from the beam index, floor((2i + 1) N_az / (2 N_b)).
 * key = b_r * N_az + b_a, or -1 when the return is not binned.
 * `ray_ids` gives the canonical index k = i * N_e + j of each ray. */
void oracle_bin_keys(const double* sd, int64_t nr, const int64_t* ray_ids, const int32_t* tri,
                     const double* t, int64_t* key)
{
    const int64_t ne = (int64_t)sd[SD_NE], nbm = (int64_t)sd[SD_NB];
    const int64_t nrb = (int64_t)sd[SD_NR], naz = (int64_t)sd[SD_NAZ];
    const double rmin = sd[SD_RMIN], rmax = sd[SD_RMAX];
    for (int64_t k = 0; k < nr; ++k) {
        key[k] = -1;
        if (tri[k] < 0) continue;
        const double r = t[k];
        if (!(r >= rmin && r < rmax)) continue;
        int64_t br = (int64_t)floor((r - rmin) * (double)nrb / (rmax - rmin));
        if (br > nrb - 1) br = nrb - 1;
        const int64_t i = ray_ids[k] / ne;
        const int64_t ba = ((2 * i + 1) * naz) / (2 * nbm);
        key[k] = br * naz + ba;
    }
}

/* P[key] += s, in canonical ray order. */
void oracle_accumulate(int64_t nr, const int64_t* key, const double* s, int64_t n_bins, double* P)
{
    memset(P, 0, sizeof(double) * (size_t)n_bins);
    for (int64_t k = 0; k < nr; ++k)
        if (key[k] >= 0) P[key[k]] += s[k];
}

/* ------------------------------------------------------------------------ */
/* Noise (Eq. 3-6)                                                           */
/* ------------------------------------------------------------------------ */

/* Range and azimuth of bin centres. */
static double bin_range(const double* sd, int64_t br)
{
    return sd[SD_RMIN] + (br + 0.5) * (sd[SD_RMAX] - sd[SD_RMIN]) / sd[SD_NR];
}
static double bin_azimuth(const double* sd, int64_t ba)
{
    return -sd[SD_HFOV] / 2.0 + (ba + 0.5) * sd[SD_HFOV] / sd[SD_NAZ];
}

void oracle_noise(const double* sd, const double* P, uint64_t seed, uint64_t frame,
                  double sigma_sa, double sigma_sm, double sigma_phi, double* Inoised)
{
    const int64_t nrb = (int64_t)sd[SD_NR], naz = (int64_t)sd[SD_NAZ];
    const double rmax = sd[SD_RMAX];
    for (int64_t br = 0; br < nrb; ++br) {
        const double rc = bin_range(sd, br);
        for (int64_t ba = 0; ba < naz; ++ba) {
            const int64_t b = br * naz + ba;
            const double phic = bin_azimuth(sd, ba);
            double w_sa, w_sm;
            bin_draws((uint64_t)b, seed, frame, sigma_sa, sigma_sm, &w_sa, &w_sm);
            const double additive = (rc * rc) / (rmax * rmax) *
                                    (1.0 + 0.5 * exp(-(phic * phic) / sigma_phi) * w_sa);   /* Eq. 3 */
            Inoised[b] = P[b] * (0.5 + w_sm) + additive;                                   /* Eq. 5 */
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Normalisation                                                             */
/* ------------------------------------------------------------------------ */

/* mode 0: none; 1: each range row divided by its maximum; 2: whole image
 * divided by its maximum.  A group whose maximum is <= 0 is left unchanged.
 * argmax[g] = lowest index attaining the maximum of group g (row-local for
 * mode 1, flat for mode 2); scale[g] = the maximum. */
void oracle_normalise(const double* sd, const double* In, int mode, double* out,
                      int64_t* argmax, double* scale)
{
    const int64_t nrb = (int64_t)sd[SD_NR], naz = (int64_t)sd[SD_NAZ];
    const int64_t n = nrb * naz;
    if (mode == 0) { memcpy(out, In, sizeof(double) * (size_t)n); return; }
    const int64_t groups = mode == 1 ? nrb : 1, len = mode == 1 ? naz : n;
    for (int64_t g = 0; g < groups; ++g) {
        const double* row = In + g * len;
        int64_t am = 0;
        for (int64_t j = 1; j < len; ++j)
            if (row[j] > row[am]) am = j;
        const double m = row[am];
        argmax[g] = am;
        scale[g] = m;
        for (int64_t j = 0; j < len; ++j) out[g * len + j] = m > 0.0 ? row[j] / m : row[j];
    }
}

/* ------------------------------------------------------------------------ */
/* Fan image                                                                 */
/* ------------------------------------------------------------------------ */

/* Square pixels, sensor at the bottom centre, the fan filling the image:
 * scale = min(W / (2 r_max sin(H/2)), Hpx / r_max) pixels per metre (H <= pi).
 * Pixel (u, v) (v = 0 at the top) has centre x = (u + 1/2 - W/2) / scale,
 * y = (Hpx - v - 1/2) / scale, r = |(x, y)|, phi = atan2(x, y).  Outside
 * r_min <= r <= r_max, |phi| <= H/2 the pixel is 0; inside it is the
 * bilinear interpolation over bin centres, clamped to the edge bins.
 * flag[p] = 1 marks pixels within 1e-5 (relative) of the fan boundary. */
void oracle_fan(const double* sd, const double* polar, int W, int Hpx, double* fan, uint8_t* flag)
{
    const int64_t nrb = (int64_t)sd[SD_NR], naz = (int64_t)sd[SD_NAZ];
    const double H = sd[SD_HFOV], rmin = sd[SD_RMIN], rmax = sd[SD_RMAX];
    const double sx = (double)W / (2.0 * rmax * sin(H / 2.0)), sy = (double)Hpx / rmax;
    const double scale = sx < sy ? sx : sy;
    const double dr = (rmax - rmin) / nrb, da = H / naz;
    for (int v = 0; v < Hpx; ++v) {
        for (int u = 0; u < W; ++u) {
            const double x = (u + 0.5 - W / 2.0) / scale;
            const double y = (Hpx - v - 0.5) / scale;
            const double r = sqrt(x * x + y * y);
            const double phi = atan2(x, y);
            const int64_t p = (int64_t)v * W + u;
            const double eps = 1e-5;
            flag[p] = (fabs(r - rmin) < eps * rmax || fabs(r - rmax) < eps * rmax ||
                       fabs(fabs(phi) - H / 2.0) < eps) ? 1 : 0;
            if (r < rmin || r > rmax || fabs(phi) > H / 2.0) { fan[p] = 0.0; continue; }
            const double fr = (r - rmin) / dr - 0.5, fa = (phi + H / 2.0) / da - 0.5;
            const double i0 = floor(fr), j0 = floor(fa);
            const double wr = fr - i0, wa = fa - j0;
            int64_t ia = (int64_t)i0, ib = ia + 1, ja = (int64_t)j0, jb = ja + 1;
            ia = ia < 0 ? 0 : (ia > nrb - 1 ? nrb - 1 : ia);
            ib = ib < 0 ? 0 : (ib > nrb - 1 ? nrb - 1 : ib);
            ja = ja < 0 ? 0 : (ja > naz - 1 ? naz - 1 : ja);
            jb = jb < 0 ? 0 : (jb > naz - 1 ? naz - 1 : jb);
            fan[p] = (1 - wr) * (1 - wa) * polar[ia * naz + ja] + (1 - wr) * wa * polar[ia * naz + jb] +
                     wr * (1 - wa) * polar[ib * naz + ja] + wr * wa * polar[ib * naz + jb];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Analytic gradient                                                         */
/* ------------------------------------------------------------------------ */

/* Given G = dL/dN (the upstream gradient of the normalised image), the
 * noised image I~ the forward produced, and the per-ray hits, returns
 * dtheta = (dL/dalpha, dL/dgain, dL/dmu[0..n_mat)).
 *   normalisation:  N_j = I~_j / m, m = I~_a (a = argmax of the group):
 *                   dL/dI~_j = G_j / m - [j = a] sum_k G_k I~_k / m^2  (m > 0)
 *   noise (Eq. 5):  dL/dP_b = dL/dI~_b (0.5 + w_sm_b)
 *   scatter-add:    each binned ray k gathers g_k = dL/dP_{key_k}
 *   intensity:      s_k = mu_m c_k e^{-2 alpha r_k} gain
 *                   dmu_m += g_k c_k e^{-2 alpha r_k} gain
 *                   dalpha += g_k s_k (-2 r_k),  dgain += g_k mu_m c_k e^{-2 alpha r_k} */
void oracle_grad(const double* sd, int mode, const double* G, const double* In,
                 uint64_t seed, uint64_t frame, double sigma_sa, double sigma_sm,
                 int64_t nr, const int64_t* key, const int32_t* tri, const double* t,
                 const double* dn, const int32_t* mat_of_tri, const double* mu, int n_mat,
                 double alpha, double gain, int two_sided, double* dtheta)
{
    const int64_t nrb = (int64_t)sd[SD_NR], naz = (int64_t)sd[SD_NAZ];
    const int64_t n = nrb * naz;
    double* gI = (double*)malloc(sizeof(double) * (size_t)n);
    if (mode == 0) {
        memcpy(gI, G, sizeof(double) * (size_t)n);
    } else {
        const int64_t groups = mode == 1 ? nrb : 1, len = mode == 1 ? naz : n;
        for (int64_t g = 0; g < groups; ++g) {
            const double* row = In + g * len;
            int64_t am = 0;
            for (int64_t j = 1; j < len; ++j)
                if (row[j] > row[am]) am = j;
            const double m = row[am];
            if (!(m > 0.0)) {
                for (int64_t j = 0; j < len; ++j) gI[g * len + j] = G[g * len + j];
                continue;
            }
            double dot = 0.0;
            for (int64_t j = 0; j < len; ++j) dot += G[g * len + j] * row[j];
            for (int64_t j = 0; j < len; ++j) gI[g * len + j] = G[g * len + j] / m;
            gI[g * len + am] -= dot / (m * m);
        }
    }
    for (int64_t b = 0; b < n; ++b) {
        double w_sa, w_sm;
        bin_draws((uint64_t)b, seed, frame, sigma_sa, sigma_sm, &w_sa, &w_sm);
        gI[b] *= 0.5 + w_sm;
    }
    for (int i = 0; i < n_mat + 2; ++i) dtheta[i] = 0.0;
    for (int64_t k = 0; k < nr; ++k) {
        if (key[k] < 0) continue;
        const double g = gI[key[k]];
        const int m = mat_of_tri[tri[k]];
        const double c = incidence(dn[k], two_sided);
        const double att = exp(-2.0 * alpha * t[k]);
        const double s = mu[m] * c * att * gain;
        dtheta[0] += g * s * (-2.0 * t[k]);
        dtheta[1] += g * mu[m] * c * att;
        dtheta[2 + m] += g * c * att * gain;
    }
    free(gI);
}

/* ------------------------------------------------------------------------ */
/* Underwater image formation (Sec. III-A-1, Eq. 1)                          */
/* ------------------------------------------------------------------------ */

/* For every pixel k and colour channel c:
 *   I_c = J_c exp(-beta_attn,c d) + B_inf,c (1 - exp(-beta_bs,c d)).
 * J: [n][3] (in-air image, pixel-major RGB), d: [n] depth in metres,
 * coef: beta_attn (R, G, B), beta_bs (R, G, B), B_inf (R, G, B).
 * A coefficient of 0 means no attenuation at any depth, also d = +inf (the
 * exponent is taken as 0 rather than 0 * inf). */
static double uw_transmission(double beta, double d)
{
    return beta == 0.0 ? 1.0 : exp(-beta * d);
}

void oracle_uw_image(const float* J, const float* d, int64_t n, const double coef[9], double* I)
{
    for (int64_t k = 0; k < n; ++k) {
        for (int c = 0; c < 3; ++c) {
            const double attn = uw_transmission(coef[c], (double)d[k]);
            const double bs = uw_transmission(coef[3 + c], (double)d[k]);
            I[3 * k + c] = (double)J[3 * k + c] * attn + coef[6 + c] * (1.0 - bs);   /* Eq. 1 */
        }
    }
}

/* ------------------------------------------------------------------------ */
/* DVL (Sec. III-A-3): four-beam convex Janus array, range-dependent rate,   */
/* dropout.  The paper fixes no geometry, rate law or noise; the readings    */
/* are: beam k (k = 0..3) points tilt off the sensor's down axis at azimuth  */
/* 45 + 90 k degrees, (sin tilt cos a_k, sin tilt sin a_k, -cos tilt) in the  */
/* sensor frame; a beam is valid when its closest hit lies in [r_min, r_max]; */
/* each valid beam measures its radial velocity b_k . v + sigma_b w_k (v the  */
/* sensor-frame velocity, w_k standard normal); the velocity is the least-    */
/* squares fit over the valid beams, reported when at least min_beams are     */
/* valid; the ping period is t0 + t1 * (farthest valid range), or t_lost when */
/* the velocity is invalid.                                                   */
/* ------------------------------------------------------------------------ */

static void dvl_beam_sensor(double tilt, int k, double b[3])
{
    const double a = M_PI / 4.0 + k * (M_PI / 2.0);
    b[0] = sin(tilt) * cos(a);
    b[1] = sin(tilt) * sin(a);
    b[2] = -cos(tilt);
}

/* World directions of the four beams of n poses (R: sensor->world, row-major). */
void oracle_dvl_beams(const double* R, int64_t n, double tilt, double* dirs)
{
    for (int64_t p = 0; p < n; ++p) {
        for (int k = 0; k < 4; ++k) {
            double b[3];
            dvl_beam_sensor(tilt, k, b);
            for (int a = 0; a < 3; ++a)
                dirs[12 * p + 3 * k + a] = R[9 * p + 3 * a] * b[0] + R[9 * p + 3 * a + 1] * b[1] +
                                           R[9 * p + 3 * a + 2] * b[2];
        }
    }
}

/* The four standard-normal beam draws of pose p: Philox4x32-10, key = seed,
 * counter (p lo, p hi, 2, h) for h = 0, 1; words (0, 1) -> beam 2h and words
 * (2, 3) -> beam 2h + 1, each by the cosine branch of Box-Muller. */
static void dvl_normals(uint64_t p, uint64_t seed, double w[4])
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 2u, h};
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        w[2 * h] = sqrt(-2.0 * log(u01(x[0]))) * cos(2.0 * M_PI * u01(x[1]));
        w[2 * h + 1] = sqrt(-2.0 * log(u01(x[2]))) * cos(2.0 * M_PI * u01(x[3]));
    }
}

/* Solves the 3x3 system A x = y by Gaussian elimination with partial pivoting. */
static int solve3(double A[3][3], double y[3], double x[3])
{
    int piv[3] = {0, 1, 2};
    for (int c = 0; c < 3; ++c) {
        int best = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[piv[r]][c]) > fabs(A[piv[best]][c])) best = r;
        const int t = piv[c]; piv[c] = piv[best]; piv[best] = t;
        const double d = A[piv[c]][c];
        if (d == 0.0) return 0;
        for (int r = c + 1; r < 3; ++r) {
            const double f = A[piv[r]][c] / d;
            for (int k = c; k < 3; ++k) A[piv[r]][k] -= f * A[piv[c]][k];
            y[piv[r]] -= f * y[piv[c]];
        }
    }
    for (int c = 2; c >= 0; --c) {
        double s = y[piv[c]];
        for (int k = c + 1; k < 3; ++k) s -= A[piv[c]][k] * x[k];
        x[c] = s / A[piv[c]][c];
    }
    return 1;
}

/* One measurement per pose.  t: [n][4] closest-hit distances along the unit
 * beams (+inf for a miss); v_world: [n][3].  Out: vel [n][3] (sensor frame, 0
 * when invalid), flags [n] (bit k: beam k valid; bit 4: velocity valid),
 * period [n] (s). */
void oracle_dvl_measure(int64_t n, const double* R, const double* v_world, const double* t, double tilt,
                        double r_min, double r_max, int min_beams, double sigma_b, double t0, double t1,
                        double t_lost, uint64_t seed, double* vel, int32_t* flags, double* period)
{
    for (int64_t p = 0; p < n; ++p) {
        double vs[3];
        for (int a = 0; a < 3; ++a)   /* R^T v: world -> sensor */
            vs[a] = R[9 * p + a] * v_world[3 * p] + R[9 * p + 3 + a] * v_world[3 * p + 1] +
                    R[9 * p + 6 + a] * v_world[3 * p + 2];
        double w[4];
        dvl_normals((uint64_t)p, seed, w);
        double A[3][3] = {{0}}, y[3] = {0};
        int nvalid = 0, f = 0;
        double far = 0.0;
        for (int k = 0; k < 4; ++k) {
            const double r = t[4 * p + k];
            if (!(r >= r_min && r <= r_max)) continue;
            f |= 1 << k;
            ++nvalid;
            if (r > far) far = r;
            double b[3];
            dvl_beam_sensor(tilt, k, b);
            const double u = b[0] * vs[0] + b[1] * vs[1] + b[2] * vs[2] + sigma_b * w[k];
            for (int i = 0; i < 3; ++i) {
                y[i] += b[i] * u;
                for (int j = 0; j < 3; ++j) A[i][j] += b[i] * b[j];
            }
        }
        double x[3] = {0, 0, 0};
        if (nvalid >= min_beams && solve3(A, y, x)) f |= 16;
        else x[0] = x[1] = x[2] = 0.0;
        for (int a = 0; a < 3; ++a) vel[3 * p + a] = x[a];
        flags[p] = f;
        period[p] = (f & 16) ? t0 + t1 * far : t_lost;
    }
}

/* Emission schedule of n_veh vehicles of n_steps steps each (period [veh][step],
 * step dt): a measurement at step 0, then at step s + max(1, ceil(period[s] / dt))
 * after a measurement at step s.  emit [veh][step] = 1 at measurement steps. */
void oracle_dvl_schedule(int64_t n_veh, int64_t n_steps, const double* period, double dt, int32_t* emit)
{
    for (int64_t v = 0; v < n_veh; ++v) {
        for (int64_t s = 0; s < n_steps; ++s) emit[v * n_steps + s] = 0;
        int64_t s = 0;
        while (s < n_steps) {
            emit[v * n_steps + s] = 1;
            double q = ceil(period[v * n_steps + s] / dt);
            if (q < 1.0) q = 1.0;
            s += (int64_t)q;
        }
    }
}
