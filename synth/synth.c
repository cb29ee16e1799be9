/*
 * Seeded synthetic HI-like spectral cube generator (input data only).
 *
 * This module produces the workloads that both the FP64 oracle and the CUDA
 * renderer consume.  It holds none of the rendering method's arithmetic: no
 * ray, sampling, transfer-function or compositing code lives here.
 *
 * A cube is RA x Dec x channel = (nx, ny, nz), stored x-fastest.  Each voxel
 * value is, evaluated in double precision and rounded once to float:
 *
 *     noise(x,y,z) + ripple(z) + sum_s source_s(x,y,z)
 *
 *   noise  : i.i.d. Gaussian, sigma from the parameters, drawn by a
 *            counter-based generator (splitmix64 finaliser keyed by the seed
 *            and the global voxel index; Box-Muller with libm, whose two
 *            outputs serve the voxel pair 2m, 2m + 1 of the linear index), so
 *            any region of the cube can be produced independently and
 *            bit-identically.
 *   ripple : ripple_amp * sigma * sin(2 pi (z + 1/2) / ripple_period + phi),
 *            phi seeded; the same for every (x, y).  A smooth continuum
 *            residual along the channel axis.
 *   source : amp * exp(-((x-cx)^2 + (y-cy)^2) / (2 s_s^2) - (z-cz)^2 / (2 s_z^2)),
 *            evaluated at voxel centres (i + 1/2), truncated at +-trunc
 *            standard deviations per axis; s = FWHM / (2 sqrt(2 ln 2)).
 *            Amplitude, spatial FWHM, spectral FWHM and centre are uniform in
 *            the configured ranges.  Sources are added in index order.
 */
#define _GNU_SOURCE /* sincos */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t nx, ny, nz;
    uint64_t seed;
    double sigma;          /* noise standard deviation                     */
    int32_t nsrc;          /* number of Gaussian sources                    */
    int32_t pad_;
    double amp_lo, amp_hi; /* source amplitude range, in units of sigma     */
    double fwhm_s_lo, fwhm_s_hi; /* spatial FWHM range, voxels              */
    double fwhm_z_lo, fwhm_z_hi; /* spectral FWHM range, channels           */
    double ripple_amp;     /* ripple amplitude in units of sigma (0 = none) */
    double ripple_period;  /* ripple period in channels                      */
    double trunc;          /* truncation radius in standard deviations      */
} syn_params;

typedef struct {
    double amp, cx, cy, cz, sig_s, sig_z;
} syn_source;

static inline uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Key of stream `stream` of a seed; uniform double in [0, 1) from (key, counter). */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream)
{
    return mix64(seed ^ (stream * 0xD1B54A32D192ED03ull));
}

static inline double uni_k(uint64_t key, uint64_t ctr)
{
    return (double)(mix64(key + ctr) >> 11) * (1.0 / 9007199254740992.0);
}

static inline double uni(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return uni_k(stream_key(seed, stream), ctr);
}

static const double TWO_PI = 6.283185307179586476925286766559;

/* Noise of voxels 2m and 2m + 1: both outputs of one Box-Muller transform of the
 * uniforms at counters 4m and 4m + 1 of stream 0 (key). */
static inline void noise_pair(uint64_t key, uint64_t m, double* n0, double* n1)
{
    const double u1 = 1.0 - uni_k(key, 4 * m); /* (0, 1] */
    const double u2 = uni_k(key, 4 * m + 1);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincos(TWO_PI * u2, &sn, &cs);
    *n0 = r * cs;
    *n1 = r * sn;
}

int syn_sources(const syn_params* p, syn_source* out)
{
    const double k = 2.0 * sqrt(2.0 * log(2.0));
    for (int s = 0; s < p->nsrc; ++s) {
        uint64_t c = (uint64_t)s * 8;
        double ua = uni(p->seed, 1, c + 0), us = uni(p->seed, 1, c + 1);
        double uz = uni(p->seed, 1, c + 2);
        double ux = uni(p->seed, 1, c + 3), uy = uni(p->seed, 1, c + 4);
        double uc = uni(p->seed, 1, c + 5);
        out[s].amp = p->sigma * (p->amp_lo + (p->amp_hi - p->amp_lo) * ua);
        out[s].sig_s = (p->fwhm_s_lo + (p->fwhm_s_hi - p->fwhm_s_lo) * us) / k;
        out[s].sig_z = (p->fwhm_z_lo + (p->fwhm_z_hi - p->fwhm_z_lo) * uz) / k;
        out[s].cx = ux * (double)p->nx;
        out[s].cy = uy * (double)p->ny;
        out[s].cz = uc * (double)p->nz;
    }
    return 0;
}

double syn_ripple_phase(const syn_params* p)
{
    return TWO_PI * uni(p->seed, 2, 0);
}

typedef struct {
    const syn_params* p;
    const syn_source* src;
    int64_t x0, y0, z0, sx, sy, sz;
    float* out;
    int64_t zbeg, zend; /* plane range (relative) handled by this worker */
    double phase;
    int rc;
} job_t;

static void idx_range(double c, double sig, double trunc, int64_t lo, int64_t hi,
                      int64_t* a, int64_t* b)
{
    /* voxel centre i + 0.5 within [c - trunc*sig, c + trunc*sig], clipped to [lo, hi) */
    double r = trunc * sig;
    int64_t i0 = (int64_t)ceil(c - r - 0.5);
    int64_t i1 = (int64_t)floor(c + r - 0.5) + 1;
    if (i0 < lo) i0 = lo;
    if (i1 > hi) i1 = hi;
    *a = i0;
    *b = i1;
}

static void* worker(void* arg)
{
    job_t* j = (job_t*)arg;
    const syn_params* p = j->p;
    const uint64_t key = stream_key(p->seed, 0);
    const int64_t sx = j->sx, sy = j->sy;
    double* acc = (double*)malloc(sizeof(double) * (size_t)(sx * sy));
    double* gx = (double*)malloc(sizeof(double) * (size_t)(sx > 0 ? sx : 1));
    double* gy = (double*)malloc(sizeof(double) * (size_t)(sy > 0 ? sy : 1));
    if (!acc || !gx || !gy) {
        j->rc = -1;
        free(acc); free(gx); free(gy);
        return NULL;
    }
    for (int64_t zr = j->zbeg; zr < j->zend; ++zr) {
        const int64_t z = j->z0 + zr;
        double rip = 0.0;
        if (p->ripple_amp != 0.0)
            rip = p->ripple_amp * p->sigma *
                  sin(TWO_PI * ((double)z + 0.5) / p->ripple_period + j->phase);
        for (int64_t yr = 0; yr < sy; ++yr) {
            const int64_t y = j->y0 + yr;
            const uint64_t row = ((uint64_t)z * (uint64_t)p->ny + (uint64_t)y) * (uint64_t)p->nx;
            double* a = acc + yr * sx;
            const uint64_t i0 = row + (uint64_t)j->x0, i1 = i0 + (uint64_t)sx;
            double n0, n1;
            uint64_t i = i0;
            if (i & 1) { /* the region starts on the second voxel of a pair */
                noise_pair(key, i >> 1, &n0, &n1);
                a[0] = p->sigma * n1 + rip;
                ++i;
            }
            for (; i + 1 < i1; i += 2) {
                noise_pair(key, i >> 1, &n0, &n1);
                a[i - i0] = p->sigma * n0 + rip;
                a[i + 1 - i0] = p->sigma * n1 + rip;
            }
            if (i < i1) {
                noise_pair(key, i >> 1, &n0, &n1);
                a[i - i0] = p->sigma * n0 + rip;
            }
        }
        for (int s = 0; s < p->nsrc; ++s) {
            const syn_source* q = &j->src[s];
            int64_t za, zb, ya, yb, xa, xb;
            idx_range(q->cz, q->sig_z, p->trunc, z, z + 1, &za, &zb);
            if (za >= zb) continue;
            idx_range(q->cy, q->sig_s, p->trunc, j->y0, j->y0 + sy, &ya, &yb);
            if (ya >= yb) continue;
            idx_range(q->cx, q->sig_s, p->trunc, j->x0, j->x0 + sx, &xa, &xb);
            if (xa >= xb) continue;
            double dz = ((double)z + 0.5 - q->cz) / q->sig_z;
            double gz = q->amp * exp(-0.5 * dz * dz);
            for (int64_t x = xa; x < xb; ++x) {
                double d = ((double)x + 0.5 - q->cx) / q->sig_s;
                gx[x - xa] = exp(-0.5 * d * d);
            }
            for (int64_t y = ya; y < yb; ++y) {
                double d = ((double)y + 0.5 - q->cy) / q->sig_s;
                gy[y - ya] = exp(-0.5 * d * d);
            }
            for (int64_t y = ya; y < yb; ++y) {
                double gyz = gz * gy[y - ya];
                double* a = acc + (y - j->y0) * sx - j->x0;
                for (int64_t x = xa; x < xb; ++x) a[x] += gyz * gx[x - xa];
            }
        }
        float* o = j->out + zr * sx * sy;
        for (int64_t i = 0; i < sx * sy; ++i) o[i] = (float)acc[i];
    }
    free(acc); free(gx); free(gy);
    j->rc = 0;
    return NULL;
}

/*
 * Fill out[(zr*sy + yr)*sx + xr] with the cube values of the region
 * [x0, x0+sx) x [y0, y0+sy) x [z0, z0+sz).  The region must lie inside the
 * cube.  Returns 0 on success, -1 on bad arguments or allocation failure.
 */
int syn_region(const syn_params* p, int64_t x0, int64_t y0, int64_t z0,
               int64_t sx, int64_t sy, int64_t sz, float* out, int nthreads)
{
    if (!p || !out || sx < 0 || sy < 0 || sz < 0 || x0 < 0 || y0 < 0 || z0 < 0 ||
        x0 + sx > p->nx || y0 + sy > p->ny || z0 + sz > p->nz || p->nsrc < 0)
        return -1;
    if (sx == 0 || sy == 0 || sz == 0) return 0;
    syn_source* src = NULL;
    syn_params q = *p; /* the same cube with only the sources that reach the region */
    if (p->nsrc > 0) {
        src = (syn_source*)malloc(sizeof(syn_source) * (size_t)p->nsrc);
        if (!src) return -1;
        syn_sources(p, src);
        int32_t kept = 0;
        for (int32_t s = 0; s < p->nsrc; ++s) {
            int64_t a, b;
            idx_range(src[s].cx, src[s].sig_s, p->trunc, x0, x0 + sx, &a, &b);
            if (a >= b) continue;
            idx_range(src[s].cy, src[s].sig_s, p->trunc, y0, y0 + sy, &a, &b);
            if (a >= b) continue;
            idx_range(src[s].cz, src[s].sig_z, p->trunc, z0, z0 + sz, &a, &b);
            if (a >= b) continue;
            src[kept++] = src[s]; /* order kept: sources are still added in index order */
        }
        q.nsrc = kept;
    }
    p = &q;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > sz) nthreads = (int)sz;
    if (nthreads > 256) nthreads = 256;
    job_t jobs[256];
    pthread_t th[256];
    int started[256] = {0};
    double phase = syn_ripple_phase(p);
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (job_t){p, src, x0, y0, z0, sx, sy, sz, out,
                          sz * t / nthreads, sz * (t + 1) / nthreads, phase, 0};
    }
    for (int t = 1; t < nthreads; ++t)
        started[t] = pthread_create(&th[t], NULL, worker, &jobs[t]) == 0;
    worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            worker(&jobs[t]);  /* no thread could be created: run it here */
    }
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].rc) rc = -1;
    free(src);
    return rc;
}

/*
 * Region callback for out-of-core renderers: `user` points to a syn_cb_user
 * (parameters + worker count).  Signature: fill dst with the region
 * [x0, x0+sx) x [y0, y0+sy) x [z0, z0+sz), x fastest; 0 on success.
 */
typedef struct {
    syn_params p;
    int32_t nthreads;
    int32_t pad_;
} syn_cb_user;

int syn_region_cb(void* user, int64_t x0, int64_t y0, int64_t z0, int64_t sx, int64_t sy, int64_t sz,
                  float* dst)
{
    const syn_cb_user* u = (const syn_cb_user*)user;
    if (!u) return -1;
    return syn_region(&u->p, x0, y0, z0, sx, sy, sz, dst, u->nthreads);
}
