/*
 * FP64 CPU oracle for ray-casting volume rendering of spectral cubes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load or run this code.  It shares no
 * code, header or constant with the CUDA renderer.
 *
 * The method is the ray-casting volume renderer of Hassan, Fluke & Barnes
 * (Abstract and Sec. 1: ray casting of spectral cubes larger than one
 * machine's memory; Sec. 3: static renders of the same orientation at a
 * user-chosen output size, 5 x 5 wall of 1920 x 1080 panels).  The paper
 * gives no formulas; the discretisation below is the standard front-to-back
 * emission-absorption ray caster, written plainly in double precision:
 *
 *   1. camera ray for pixel (px, py): pixel centre, rows top-down;
 *      orthographic rays start on the image plane, perspective rays at the eye.
 *   2. slab intersection with the box [0,nx] x [0,ny] x [0,nz], t >= 0.
 *   3. samples at t_k = k * step for k = ceil(t_near/step) .. ceil(t_far/step)-1
 *      (globally aligned, half-open interval).
 *   4. trilinear interpolation, voxel (i,j,k) centred at (i+1/2, j+1/2, k+1/2),
 *      clamp-to-edge.
 *   5. transfer function: node-centred linear interpolation of an n x 4 RGBA
 *      table over [vmin, vmax], clamped outside.
 *   6. front-to-back "over": C += T a rgb, T *= (1 - a); stop after the sample
 *      at which 1 - T >= ert (early ray termination).  Output (C, 1 - T),
 *      premultiplied.  MIP: TF(max v) straight, (0,0,0,0) with no samples.
 *   7. adjoint of 6 with respect to the table entries and the voxels.
 *
 * Ambiguous rays (a decision that the renderer takes in lower precision lies
 * within its rounding of the threshold) are flagged so that a test can accept
 * either outcome.  The windows follow from the renderer's arithmetic, stated
 * here as an error model (the scene's pos_err and u = 2^-24):
 *   - each sample position is within pos_err voxels (every axis) of the exact
 *     one; every FP32 operation rounds to nearest (relative error <= u);
 *   - the ray set-up is float-float (about 44 bits): a plane crossing
 *     t = (X - o_a) / d_a is within 2^-43 (|o_a| + n_a + |t|) / |d_a| of the
 *     exact one, so t/step is within that divided by step; the window used is
 *     2^7 times wider.
 * Then (first order, each window twice the bound):
 *   bit 0: t_near/step within the set-up bound of an integer (first sample in or out)
 *   bit 1: t_far/step within it (last sample in or out)
 *   bit 2: some 1 - T within E_k of ert, where E_k bounds the FP32 error of
 *          1 - T after sample k: E_k = (1 - a_k) E_{k-1} + T_{k-1} da_k + 2 u T_k,
 *          da_k the alpha error from the sample-value error dv_k (see trilinear)
 *          through the table slope, plus the FP32 threshold's own rounding.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t type; /* 0 orthographic, 1 perspective */
    int32_t pad_;
    double eye[3], right[3], up[3], fwd[3];
    double win[4]; /* l, r, b, t */
    int32_t width, height;
} orc_camera;

typedef struct {
    int64_t nx, ny, nz;
    const float* vol; /* stored voxel values, x fastest */
    const float* tf;  /* ntf x 4 straight RGBA */
    int32_t ntf;
    int32_t mode;     /* 0 composite, 1 maximum-intensity projection */
    double vmin, vmax;
    double step;
    double ert;       /* termination threshold on accumulated alpha; > 1 disables */
    int32_t dk0, dk1; /* shifts applied to the first / end sample index (variants) */
    double pos_err;   /* error model: bound on the renderer's sample-position error, voxels */
    int32_t dstop;    /* variant: stop |dstop| samples after (> 0) or before (< 0) the
                         sample at which termination happens; 0 = none */
    int32_t pad_;
} orc_scene;

#define U32 5.9604644775390625e-08 /* 2^-24, unit roundoff of FP32 */

#define FLAG_K0 1
#define FLAG_K1 2
#define FLAG_ERT 4

/* ---------------------------------------------------------------- step 1: ray */
static void camera_ray(const orc_camera* c, int64_t px, int64_t py, double o[3], double d[3])
{
    double l = c->win[0], r = c->win[1], b = c->win[2], t = c->win[3];
    double u = l + ((double)px + 0.5) * (r - l) / (double)c->width;
    double v = t - ((double)py + 0.5) * (t - b) / (double)c->height;
    double dd[3];
    for (int a = 0; a < 3; ++a) {
        if (c->type == 0) {
            o[a] = c->eye[a] + u * c->right[a] + v * c->up[a];
            dd[a] = c->fwd[a];
        } else {
            o[a] = c->eye[a];
            dd[a] = c->fwd[a] + u * c->right[a] + v * c->up[a];
        }
    }
    double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    for (int a = 0; a < 3; ++a) d[a] = dd[a] / len;
}

/* ---------------------------------------------------------------- step 2: slab */
/* Interval [tnear, tfar) of the ray in the box, t >= 0; an_/af_ receive the axis whose
   plane sets each end (-1: tnear is the t >= 0 clamp). */
static int box_interval(const orc_scene* s, const double o[3], const double d[3],
                        double* tnear, double* tfar, int* an_, int* af_)
{
    double n[3] = {(double)s->nx, (double)s->ny, (double)s->nz};
    double lo = 0.0, hi = INFINITY;
    int an = -1, af = -1;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > n[a]) return 0;
            continue;
        }
        double t1 = (0.0 - o[a]) / d[a];
        double t2 = (n[a] - o[a]) / d[a];
        double tl = t1 < t2 ? t1 : t2, th = t1 < t2 ? t2 : t1;
        if (tl > lo) {
            lo = tl;
            an = a;
        }
        if (th < hi) {
            hi = th;
            af = a;
        }
    }
    *tnear = lo;
    *tfar = hi;
    if (an_) *an_ = an;
    if (af_) *af_ = af;
    return lo < hi;
}

/* ------------------------------------------------------------ step 4: trilinear */
static int64_t clampi(int64_t i, int64_t n)
{
    return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
}

static double voxel(const orc_scene* s, int64_t x, int64_t y, int64_t z)
{
    return (double)s->vol[(z * s->ny + y) * s->nx + x];
}

/* Value at p plus, optionally, the 8 voxel indices and weights it used, and a bound
   dv on how far the renderer's FP32 value of this sample can be from it (error model
   of the header, first order): moving the position by pos_err on each axis changes
   the value by at most pos_err * sum_a D_a, D_a the largest difference of neighbouring
   voxels along axis a around the sample (the cell's edges, taken one cell inwards at a
   clamped face so that a sample pushed across the face is covered).  The FP32 lerps
   lerp(f, a, b) = a + f (b - a), three levels (x, y, z), add at each level one
   rounding of a difference (at most u D_a) and one of a convex combination (at most
   u M, M the largest |corner|): u (sum_a D_a + 3 M) in all. */
static double trilinear(const orc_scene* s, const double p[3], int64_t idx[8], double w[8],
                        double* dv)
{
    int64_t n[3] = {s->nx, s->ny, s->nz};
    int64_t i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double q = p[a] - 0.5;
        double fl = floor(q);
        f[a] = q - fl;
        i0[a] = clampi((int64_t)fl, n[a]);
        i1[a] = clampi((int64_t)fl + 1, n[a]);
    }
    double val = 0.0, M = 0.0;
    int c = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx, ++c) {
                int64_t x = dx ? i1[0] : i0[0];
                int64_t y = dy ? i1[1] : i0[1];
                int64_t z = dz ? i1[2] : i0[2];
                double wt = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                            (dz ? f[2] : 1.0 - f[2]);
                int64_t li = (z * s->ny + y) * s->nx + x;
                val += wt * (double)s->vol[li];
                if (fabs((double)s->vol[li]) > M) M = fabs((double)s->vol[li]);
                if (idx) idx[c] = li;
                if (w) w[c] = wt;
            }
    if (dv) {
        double sumD = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (n[a] < 2) continue;
            int64_t j0 = (int64_t)floor(p[a] - 0.5);
            if (j0 < 0) j0 = 0;
            if (j0 > n[a] - 2) j0 = n[a] - 2;
            int b0 = (a + 1) % 3, b1 = (a + 2) % 3;
            double D = 0.0;
            for (int e = 0; e < 4; ++e) {
                int64_t q0[3], q1[3];
                q0[a] = j0;
                q1[a] = j0 + 1;
                q0[b0] = q1[b0] = (e & 1) ? i1[b0] : i0[b0];
                q0[b1] = q1[b1] = (e & 2) ? i1[b1] : i0[b1];
                double dd = fabs(voxel(s, q1[0], q1[1], q1[2]) - voxel(s, q0[0], q0[1], q0[2]));
                if (dd > D) D = dd;
            }
            sumD += D;
        }
        *dv = s->pos_err * sumD + U32 * (sumD + 3.0 * M);
    }
    return val;
}

/* ------------------------------------------------------- step 5: transfer function */
typedef struct {
    double rgba[4];
    int32_t i;       /* lower table entry */
    double w;        /* weight of entry i+1 */
    double slope[4]; /* d rgba / d v (0 where the lookup is clamped) */
} tf_eval_t;

static void tf_lookup(const orc_scene* s, double v, tf_eval_t* e)
{
    double u = (v - s->vmin) / (s->vmax - s->vmin);
    int inside = (u > 0.0 && u < 1.0);
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    double x = u * (double)(s->ntf - 1);
    int32_t i = (int32_t)floor(x);
    if (i > s->ntf - 2) i = s->ntf - 2;
    double w = x - (double)i;
    e->i = i;
    e->w = w;
    for (int c = 0; c < 4; ++c) {
        double a = s->tf[4 * i + c], b = s->tf[4 * (i + 1) + c];
        e->rgba[c] = (1.0 - w) * a + w * b;
        e->slope[c] = inside ? (b - a) * (double)(s->ntf - 1) / (s->vmax - s->vmin) : 0.0;
    }
}

/* Bound on the renderer's alpha error for a sample of value v whose FP32 value is
   within dv of v: the steepest alpha slope among the table segments that a value in
   [v - dv, v + dv] can reach, times dv, plus the rounding of the table position
   x = (v - vmin) (1 / (vmax - vmin)) (n - 1) (four roundings: at most 4 u (|x| + 1)
   in segment units) and of the lerp (2 u max alpha). */
static double alpha_err(const orc_scene* s, double v, double dv)
{
    double scale = (double)(s->ntf - 1) / (s->vmax - s->vmin);
    double x = (v - s->vmin) * scale;
    double xr = dv * scale + 4.0 * U32 * (fabs(x) + 1.0);
    double jlo = floor(x - xr), jhi = floor(x + xr);
    if (jlo < 0.0) jlo = 0.0;
    if (jhi > (double)(s->ntf - 2)) jhi = (double)(s->ntf - 2);
    double smax = 0.0, amax = 0.0;
    for (int64_t j = (int64_t)jlo; j <= (int64_t)jhi; ++j) {
        double a0 = s->tf[4 * j + 3], a1 = s->tf[4 * (j + 1) + 3];
        if (fabs(a1 - a0) > smax) smax = fabs(a1 - a0);
        if (fabs(a0) > amax) amax = fabs(a0);
        if (fabs(a1) > amax) amax = fabs(a1);
    }
    if (x + xr < 0.0 || x - xr > (double)(s->ntf - 1)) smax = 0.0; /* clamped: constant */
    if (jlo > jhi) { /* reach entirely outside the table: the clamped end entry */
        int64_t j = x < 0.0 ? 0 : s->ntf - 1;
        amax = fabs(s->tf[4 * j + 3]);
    }
    return smax * xr + 2.0 * U32 * amax;
}

/* A sample whose table position is within the renderer's rounding (twice the bound
   from a value error dv) of a node may take the slope of the segment on the other side
   (reading R14; at the end nodes the other side is the clamped region, slope 0).
   Returns |sum_c g_c (s_left_c - s_right_c)| for such a sample, else 0. */
static double node_alt(const orc_scene* s, double v, double dv, const double g[4])
{
    double scale = (double)(s->ntf - 1) / (s->vmax - s->vmin);
    double x = (v - s->vmin) * scale;
    double xr = 2.0 * (dv * scale + 4.0 * U32 * (fabs(x) + 1.0));
    double j = nearbyint(x);
    if (fabs(x - j) > xr || j < 0.0 || j > (double)(s->ntf - 1)) return 0.0;
    int64_t jn = (int64_t)j;
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) {
        double sl = jn > 0 ? (s->tf[4 * jn + c] - s->tf[4 * (jn - 1) + c]) * scale : 0.0;
        double sr = jn < s->ntf - 1 ? (s->tf[4 * (jn + 1) + c] - s->tf[4 * jn + c]) * scale : 0.0;
        acc += g[c] * (sl - sr);
    }
    return fabs(acc);
}

static double frac_dist(double x)
{
    return fabs(x - nearbyint(x));
}

/* Window of t/step at a slab end set by axis a: twice 2^6 times the float-float
   set-up bound 2^-43 (|o_a| + n_a + |t|) / |d_a| of the header, over step. */
static double end_window(const orc_scene* s, const double o[3], const double d[3], int a, double t)
{
    double n[3] = {(double)s->nx, (double)s->ny, (double)s->nz};
    return ldexp(1.0, -36) * (fabs(o[a]) + n[a] + fabs(t)) / (fabs(d[a]) * s->step);
}

/* Sample index range [k0, k1) of a ray and its ambiguity flags. */
static int ray_samples(const orc_scene* s, const double o[3], const double d[3],
                       int64_t* k0, int64_t* k1, int* flags)
{
    double tn, tf;
    int an, af;
    *k0 = *k1 = 0;
    if (!box_interval(s, o, d, &tn, &tf, &an, &af)) return 0;
    double a = tn / s->step, b = tf / s->step;
    if (an >= 0 && tn > 0.0 && frac_dist(a) <= end_window(s, o, d, an, tn)) *flags |= FLAG_K0;
    if (af >= 0 && frac_dist(b) <= end_window(s, o, d, af, tf)) *flags |= FLAG_K1;
    *k0 = (int64_t)ceil(a) + s->dk0;
    *k1 = (int64_t)ceil(b) + s->dk1;
    if (*k0 < 0) *k0 = 0;
    return *k1 > *k0;
}

/* ------------------------------------------------------------- steps 3 and 6: march */
typedef struct {
    double rgba[4];
    double vmax;     /* maximum sample value (MIP), -inf with no samples */
    int64_t nsamp;   /* samples executed */
    int flags;
} ray_result;

static void trace(const orc_scene* s, const orc_camera* cam, int64_t px, int64_t py,
                  ray_result* r)
{
    double o[3], d[3];
    int64_t k0, k1;
    memset(r, 0, sizeof(*r));
    r->vmax = -INFINITY;
    camera_ray(cam, px, py, o, d);
    if (!ray_samples(s, o, d, &k0, &k1, &r->flags)) return;
    const int ert_on = s->mode == 0 && s->ert <= 1.0;
    int64_t nstop = -1; /* variant: execute exactly this many samples */
    if (ert_on && s->dstop != 0) {
        orc_scene s0 = *s;
        s0.dstop = 0;
        ray_result r0;
        trace(&s0, cam, px, py, &r0);
        nstop = r0.nsamp + s->dstop;
        if (nstop < 1) nstop = 1;
    }
    /* the renderer tests 1 - T >= ert with ert and 1 - T rounded to FP32 */
    const double ert_win = fabs(s->ert - (double)(float)s->ert) + 2.0 * U32;
    double C[3] = {0, 0, 0}, T = 1.0, m = -INFINITY, E = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
        double t = (double)k * s->step;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        double dv;
        double v = trilinear(s, p, NULL, NULL, &dv);
        r->nsamp++;
        if (s->mode == 1) {
            if (v > m) m = v;
            continue;
        }
        tf_eval_t e;
        tf_lookup(s, v, &e);
        double a = e.rgba[3];
        for (int c = 0; c < 3; ++c) C[c] += T * a * e.rgba[c];
        double Tn = T * (1.0 - a);
        E = fabs(1.0 - a) * E + T * alpha_err(s, v, dv) + 2.0 * U32 * fabs(Tn);
        T = Tn;
        if (nstop >= 0) {
            if (r->nsamp == nstop) break;
            continue;
        }
        if (ert_on && fabs((1.0 - T) - s->ert) <= 2.0 * E + ert_win) r->flags |= FLAG_ERT;
        if (ert_on && 1.0 - T >= s->ert) break;
    }
    if (s->mode == 1) {
        r->vmax = m;
        tf_eval_t e;
        tf_lookup(s, m, &e);
        for (int c = 0; c < 4; ++c) r->rgba[c] = e.rgba[c];
    } else {
        for (int c = 0; c < 3; ++c) r->rgba[c] = C[c];
        r->rgba[3] = 1.0 - T;
    }
}

/* ---------------------------------------------------------------- threading */
typedef struct {
    const orc_scene* s;
    const orc_camera* cam;
    const int64_t* pix; /* flat pixel indices py*W+px, or NULL for all */
    int64_t npix;
    double* out_rgba;
    double* out_max;
    int64_t* out_ns;
    int32_t* out_flags;
    int64_t next;       /* shared work counter */
    pthread_mutex_t mu;
    int64_t brick;      /* >0: sort-last by bricks of this edge */
} render_job;

static int64_t grab(render_job* j, int64_t chunk)
{
    pthread_mutex_lock(&j->mu);
    int64_t i = j->next;
    j->next += chunk;
    pthread_mutex_unlock(&j->mu);
    return i;
}

static void trace_sortlast(const orc_scene* s, const orc_camera* cam, int64_t B, int64_t px,
                           int64_t py, ray_result* r);

static void* render_worker(void* arg)
{
    render_job* j = (render_job*)arg;
    const int64_t chunk = 64;
    for (;;) {
        int64_t i0 = grab(j, chunk);
        if (i0 >= j->npix) break;
        int64_t i1 = i0 + chunk < j->npix ? i0 + chunk : j->npix;
        for (int64_t i = i0; i < i1; ++i) {
            int64_t flat = j->pix ? j->pix[i] : i;
            int64_t px = flat % j->cam->width, py = flat / j->cam->width;
            ray_result r;
            if (j->brick > 0)
                trace_sortlast(j->s, j->cam, j->brick, px, py, &r);
            else
                trace(j->s, j->cam, px, py, &r);
            for (int c = 0; c < 4; ++c) j->out_rgba[4 * i + c] = r.rgba[c];
            if (j->out_max) j->out_max[i] = r.vmax;
            if (j->out_ns) j->out_ns[i] = r.nsamp;
            if (j->out_flags) j->out_flags[i] = r.flags;
        }
    }
    return NULL;
}

static int run_threads(void* (*fn)(void*), void* arg, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t th[512];
    int started[512] = {0};
    for (int t = 1; t < nthreads; ++t) started[t] = pthread_create(&th[t], NULL, fn, arg) == 0;
    fn(arg);
    for (int t = 1; t < nthreads; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    return 0;
}

static int scene_ok(const orc_scene* s)
{
    return s && s->vol && s->tf && s->nx > 0 && s->ny > 0 && s->nz > 0 && s->ntf >= 2 &&
           s->step > 0.0 && s->vmax > s->vmin;
}

/*
 * Render the listed pixels (flat index py*width+px; pix == NULL renders all
 * width*height pixels in order).  out_rgba: npix x 4; out_max, out_ns,
 * out_flags: npix each, may be NULL.  Returns 0, or -1 on bad arguments.
 */
int orc_render(const orc_scene* s, const orc_camera* cam, const int64_t* pix, int64_t npix,
               double* out_rgba, double* out_max, int64_t* out_ns, int32_t* out_flags,
               int nthreads)
{
    if (!scene_ok(s) || !cam || !out_rgba || cam->width <= 0 || cam->height <= 0) return -1;
    if (!pix) npix = (int64_t)cam->width * cam->height;
    render_job j = {s, cam, pix, npix, out_rgba, out_max, out_ns, out_flags, 0,
                    PTHREAD_MUTEX_INITIALIZER, 0};
    run_threads(render_worker, &j, nthreads);
    return 0;
}

/* ------------------------------------------------------------- sort-last form */
/*
 * The same samples, grouped by the B^3 brick containing each sample position
 * (floor(p/B), clamped to the brick grid).  Each brick's samples form a
 * partial result starting from T = 1 (no termination inside a partial); the
 * partials are folded with "over" (or max) in the visibility order of the
 * bricks: ascending sum over axes of |b - e|, e = brick index of the eye
 * (perspective) or ascending sum of sign(d) * b (orthographic), ties by
 * linear brick index.  The fold stops after the partial at which 1 - T >=
 * ert, which is exact only for ert > 1.
 */
typedef struct {
    int64_t key, id;
    double C[3], T, m;
} partial_t;

static int cmp_partial(const void* a, const void* b)
{
    const partial_t* x = (const partial_t*)a;
    const partial_t* y = (const partial_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

static void trace_sortlast(const orc_scene* s, const orc_camera* cam, int64_t B, int64_t px,
                           int64_t py, ray_result* r)
{
    double o[3], d[3];
    int64_t k0, k1;
    memset(r, 0, sizeof(*r));
    r->vmax = -INFINITY;
    camera_ray(cam, px, py, o, d);
    if (!ray_samples(s, o, d, &k0, &k1, &r->flags)) return;
    int64_t nb[3] = {(s->nx + B - 1) / B, (s->ny + B - 1) / B, (s->nz + B - 1) / B};
    int64_t e[3];
    for (int a = 0; a < 3; ++a) e[a] = (int64_t)floor(cam->eye[a] / (double)B);
    int64_t cap = 64, np = 0;
    partial_t* P = (partial_t*)malloc(sizeof(partial_t) * (size_t)cap);
    for (int64_t k = k0; k < k1; ++k) {
        double t = (double)k * s->step;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        int64_t b[3];
        for (int a = 0; a < 3; ++a) {
            b[a] = (int64_t)floor(p[a] / (double)B);
            if (b[a] < 0) b[a] = 0;
            if (b[a] > nb[a] - 1) b[a] = nb[a] - 1;
        }
        int64_t id = (b[2] * nb[1] + b[1]) * nb[0] + b[0];
        partial_t* q = NULL;
        for (int64_t i = 0; i < np; ++i)
            if (P[i].id == id) q = &P[i];
        if (!q) {
            if (np == cap) {
                cap *= 2;
                P = (partial_t*)realloc(P, sizeof(partial_t) * (size_t)cap);
            }
            q = &P[np++];
            q->id = id;
            q->key = 0;
            for (int a = 0; a < 3; ++a) {
                if (cam->type == 1)
                    q->key += b[a] > e[a] ? b[a] - e[a] : e[a] - b[a];
                else
                    q->key += d[a] > 0 ? b[a] : (d[a] < 0 ? -b[a] : 0);
            }
            q->C[0] = q->C[1] = q->C[2] = 0.0;
            q->T = 1.0;
            q->m = -INFINITY;
        }
        double v = trilinear(s, p, NULL, NULL, NULL);
        r->nsamp++;
        if (v > q->m) q->m = v;
        if (s->mode == 0) {
            tf_eval_t ev;
            tf_lookup(s, v, &ev);
            double a = ev.rgba[3];
            for (int c = 0; c < 3; ++c) q->C[c] += q->T * a * ev.rgba[c];
            q->T *= (1.0 - a);
        }
    }
    qsort(P, (size_t)np, sizeof(partial_t), cmp_partial);
    double C[3] = {0, 0, 0}, T = 1.0, m = -INFINITY;
    for (int64_t i = 0; i < np; ++i) {
        if (P[i].m > m) m = P[i].m;
        if (s->mode == 0) {
            for (int c = 0; c < 3; ++c) C[c] += T * P[i].C[c];
            T *= P[i].T;
            if (s->ert <= 1.0 && 1.0 - T >= s->ert) break;
        }
    }
    free(P);
    if (s->mode == 1) {
        r->vmax = m;
        tf_eval_t ev;
        tf_lookup(s, m, &ev);
        for (int c = 0; c < 4; ++c) r->rgba[c] = ev.rgba[c];
    } else {
        for (int c = 0; c < 3; ++c) r->rgba[c] = C[c];
        r->rgba[3] = 1.0 - T;
    }
}

int orc_render_sortlast(const orc_scene* s, const orc_camera* cam, int64_t brick,
                        const int64_t* pix, int64_t npix, double* out_rgba, double* out_max,
                        int nthreads)
{
    if (!scene_ok(s) || !cam || !out_rgba || brick <= 0) return -1;
    if (!pix) npix = (int64_t)cam->width * cam->height;
    render_job j = {s, cam, pix, npix, out_rgba, out_max, NULL, NULL, 0,
                    PTHREAD_MUTEX_INITIALIZER, brick};
    run_threads(render_worker, &j, nthreads);
    return 0;
}

/* ------------------------------------------------- per-brick partial images */
/*
 * The partial image of one brick (the paper's parts of a cube rendered apart
 * and combined, Abstract and Sec. 1): for each listed pixel, the ray's samples
 * owned by brick `brick` of the B^3 decomposition (the brick containing the
 * sample position, floor(p/B) clamped to the brick grid, as in the sort-last
 * form above) composited front to back from T = 1 with no termination, as
 * (C, T) -- premultiplied colour and transmittance -- plus their maximum (MIP)
 * and count.  Folding the bricks' partials per pixel in ascending visibility
 * key (ties by brick id) with C += T C_b, T *= T_b gives orc_render_sortlast.
 * out_ct: npix x 4 (C0, C1, C2, T); out_max, out_ns: npix each (may be NULL);
 * out_key receives the brick's visibility key.  Returns 0, or -1 on bad arguments.
 */
int orc_brick_partial(const orc_scene* s, const orc_camera* cam, int64_t B, int64_t brick,
                      const int64_t* pix, int64_t npix, double* out_ct, double* out_max,
                      int64_t* out_ns, int64_t* out_key)
{
    if (!scene_ok(s) || !cam || !pix || !out_ct || !out_key || B <= 0) return -1;
    int64_t nb[3] = {(s->nx + B - 1) / B, (s->ny + B - 1) / B, (s->nz + B - 1) / B};
    if (brick < 0 || brick >= nb[0] * nb[1] * nb[2]) return -1;
    int64_t bb[3] = {brick % nb[0], (brick / nb[0]) % nb[1], brick / (nb[0] * nb[1])};
    int64_t key = 0;
    for (int64_t i = 0; i < npix; ++i) {
        int64_t px = pix[i] % cam->width, py = pix[i] / cam->width;
        double o[3], d[3];
        int64_t k0, k1;
        int flags = 0;
        camera_ray(cam, px, py, o, d);
        double C[3] = {0, 0, 0}, T = 1.0, m = -INFINITY;
        int64_t n = 0;
        if (ray_samples(s, o, d, &k0, &k1, &flags)) {
            for (int64_t k = k0; k < k1; ++k) {
                double t = (double)k * s->step;
                double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                int inside = 1;
                for (int a = 0; a < 3; ++a) {
                    int64_t b = (int64_t)floor(p[a] / (double)B);
                    if (b < 0) b = 0;
                    if (b > nb[a] - 1) b = nb[a] - 1;
                    if (b != bb[a]) inside = 0;
                }
                if (!inside) continue;
                double v = trilinear(s, p, NULL, NULL, NULL);
                ++n;
                if (v > m) m = v;
                tf_eval_t e;
                tf_lookup(s, v, &e);
                double a = e.rgba[3];
                for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * e.rgba[ch];
                T *= (1.0 - a);
            }
        }
        for (int c = 0; c < 3; ++c) out_ct[4 * i + c] = C[c];
        out_ct[4 * i + 3] = T;
        if (out_max) out_max[i] = m;
        if (out_ns) out_ns[i] = n;
    }
    /* visibility key of the brick, as in trace_sortlast */
    int64_t e[3];
    for (int a = 0; a < 3; ++a) e[a] = (int64_t)floor(cam->eye[a] / (double)B);
    double c0[3];
    if (cam->type == 0) {
        double o[3];
        camera_ray(cam, 0, 0, o, c0);
    }
    for (int a = 0; a < 3; ++a) {
        if (cam->type == 1)
            key += bb[a] > e[a] ? bb[a] - e[a] : e[a] - bb[a];
        else
            key += c0[a] > 0 ? bb[a] : (c0[a] < 0 ? -bb[a] : 0);
    }
    *out_key = key;
    return 0;
}

/* ------------------------------------------------------------- step 7: adjoint */
typedef struct {
    int64_t k;        /* sample index */
    double T;         /* transmittance before the sample */
    double a, rgb[3];
    double v, dv;     /* value, and the bound on the renderer's error in it */
    tf_eval_t e;
    int64_t idx[8];
    double w[8];
} rec_t;

/* Per-ray scratch of the adjoint: the executed samples of the ray and of one variant,
   and dL/dv per sample for both. */
typedef struct {
    rec_t* buf[2];
    double* dvs[2];
    double* alt;
    int64_t cap[2];
} ray_work;

static void work_reserve(ray_work* w, int b, int64_t n)
{
    if (n <= w->cap[b]) return;
    int64_t c = w->cap[b] ? w->cap[b] : 256;
    while (c < n) c *= 2;
    w->buf[b] = (rec_t*)realloc(w->buf[b], sizeof(rec_t) * (size_t)c);
    w->dvs[b] = (double*)realloc(w->dvs[b], sizeof(double) * (size_t)c);
    if (b == 0) w->alt = (double*)realloc(w->alt, sizeof(double) * (size_t)c);
    w->cap[b] = c;
}

/* Forward march of samples k0 .. k1-1 recording each executed one: composite stops
   after the sample at which 1 - T >= ert, or after exactly nstop samples when
   nstop >= 0; MIP records every sample.  Returns the number recorded. */
static int64_t fwd_records(const orc_scene* s, const double o[3], const double d[3], int64_t k0,
                           int64_t k1, int64_t nstop, ray_work* w, int b)
{
    int64_t n = 0;
    double T = 1.0;
    for (int64_t k = k0; k < k1; ++k) {
        work_reserve(w, b, n + 1);
        rec_t* q = &w->buf[b][n++];
        double t = (double)k * s->step;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        q->k = k;
        q->v = trilinear(s, p, q->idx, q->w, &q->dv);
        tf_lookup(s, q->v, &q->e);
        if (s->mode == 1) continue;
        q->T = T;
        q->a = q->e.rgba[3];
        for (int c = 0; c < 3; ++c) q->rgb[c] = q->e.rgba[c];
        T *= (1.0 - q->a);
        if (nstop >= 0) {
            if (n == nstop) break;
        } else if (s->ert <= 1.0 && 1.0 - T >= s->ert) {
            break;
        }
    }
    return n;
}

/* Index of the first sample attaining the maximum value (MIP), -1 with no samples. */
static int64_t first_max(const rec_t* q, int64_t n)
{
    int64_t km = -1;
    double m = -INFINITY;
    for (int64_t k = 0; k < n; ++k)
        if (q[k].v > m) {
            m = q[k].v;
            km = k;
        }
    return km;
}

/* Reverse sweep over the n recorded samples for dL/dI = g: dL/dv of each sample into
   dvs, the table gradient added to dtf (when not NULL), and into alt (when not NULL)
   the node alternative of each sample (node_alt: how much dL/dv changes if the table
   slope of the other side of a nearby node is taken). */
static void rev_sweep(const orc_scene* s, const rec_t* buf, int64_t n, const double g[4],
                      double* dtf, double* dvs, double* alt)
{
    for (int64_t k = 0; k < n; ++k) {
        dvs[k] = 0.0;
        if (alt) alt[k] = 0.0;
    }
    if (s->mode == 1) {
        /* I = TF(max v): the gradient reaches the first maximal sample only */
        int64_t km = first_max(buf, n);
        if (km < 0) return;
        const tf_eval_t* e = &buf[km].e;
        double dv = 0.0;
        for (int c = 0; c < 4; ++c) {
            if (dtf) {
                dtf[4 * e->i + c] += (1.0 - e->w) * g[c];
                dtf[4 * (e->i + 1) + c] += e->w * g[c];
            }
            dv += g[c] * e->slope[c];
        }
        dvs[km] = dv;
        if (alt) alt[km] = node_alt(s, buf[km].v, buf[km].dv, g);
        return;
    }
    /* R = colour composited behind the sample (starting from T = 1),
       P = transmittance behind the sample */
    double R[3] = {0, 0, 0}, P = 1.0;
    for (int64_t k = n - 1; k >= 0; --k) {
        const rec_t* q = &buf[k];
        double ga = g[3] * q->T * P;
        double gc[3];
        for (int c = 0; c < 3; ++c) {
            gc[c] = g[c] * q->T * q->a;
            ga += g[c] * q->T * (q->rgb[c] - R[c]);
        }
        for (int c = 0; c < 3; ++c) R[c] = q->a * q->rgb[c] + (1.0 - q->a) * R[c];
        P *= (1.0 - q->a);
        double gch[4] = {gc[0], gc[1], gc[2], ga};
        double dv = 0.0;
        for (int c = 0; c < 4; ++c) {
            if (dtf) {
                dtf[4 * q->e.i + c] += (1.0 - q->e.w) * gch[c];
                dtf[4 * (q->e.i + 1) + c] += q->e.w * gch[c];
            }
            dv += gch[c] * q->e.slope[c];
        }
        dvs[k] = dv;
        if (alt) alt[k] = node_alt(s, q->v, q->dv, gch);
    }
}

static void add_amb(double* amb, const rec_t* q, double x)
{
    for (int c = 0; c < 8; ++c) amb[q->idx[c]] += q->w[c] * x;
}

/* Adjoint of one ray.  With amb, also a per-voxel bound on how far the renderer may
   legitimately be from dvol (readings R11, R14, R15): for every sample near a table
   node, its node alternative; for MIP, every sample whose value is within the
   renderer's rounding of the maximum (either may be the first maximal one); for a
   flagged ray (an end sample or the termination within rounding), the difference of
   each sample's dL/dv between the ray and each alternative outcome. */
static void ray_backward(const orc_scene* s, const orc_camera* cam, int64_t px, int64_t py,
                         const double g[4], double* dtf, double* dvol, double* amb, ray_work* w)
{
    double o[3], d[3];
    int64_t k0, k1;
    int flags = 0;
    camera_ray(cam, px, py, o, d);
    if (!ray_samples(s, o, d, &k0, &k1, &flags)) return;
    int64_t n = fwd_records(s, o, d, k0, k1, -1, w, 0);
    rev_sweep(s, w->buf[0], n, g, dtf, w->dvs[0], amb ? w->alt : NULL);
    if (dvol)
        for (int64_t k = 0; k < n; ++k)
            for (int c = 0; c < 8; ++c) dvol[w->buf[0][k].idx[c]] += w->buf[0][k].w[c] * w->dvs[0][k];
    if (!amb) return;
    for (int64_t k = 0; k < n; ++k)
        if (w->alt[k] > 0.0) add_amb(amb, &w->buf[0][k], w->alt[k]);
    if (s->mode == 1) {
        int64_t km = first_max(w->buf[0], n);
        if (km >= 0) {
            const rec_t* qm = &w->buf[0][km];
            double gm = fabs(w->dvs[0][km]);
            int tie = 0;
            for (int64_t k = 0; k < n; ++k)
                if (k != km && w->buf[0][k].v >= qm->v - 2.0 * (w->buf[0][k].dv + qm->dv)) {
                    add_amb(amb, &w->buf[0][k], gm);
                    tie = 1;
                }
            if (tie) add_amb(amb, qm, gm);
        }
    }
    ray_result rr;
    trace(s, cam, px, py, &rr);
    if (!rr.flags) return;
    const int dk0s[3] = {0, -1, 1}, dk1s[3] = {0, -1, 1}, dss[3] = {0, -1, 1};
    int nk0 = (rr.flags & FLAG_K0) ? 3 : 1, nk1 = (rr.flags & FLAG_K1) ? 3 : 1;
    int nds = (rr.flags & FLAG_ERT) ? 3 : 1;
    for (int i0 = 0; i0 < nk0; ++i0)
        for (int i1 = 0; i1 < nk1; ++i1)
            for (int id = 0; id < nds; ++id) {
                if (i0 == 0 && i1 == 0 && id == 0) continue;
                int64_t a0 = k0 + dk0s[i0], a1 = k1 + dk1s[i1];
                if (a0 < 0) a0 = 0;
                int64_t nv = 0;
                if (a1 > a0) {
                    int64_t nstop = -1;
                    if (dss[id] != 0) {
                        nstop = fwd_records(s, o, d, a0, a1, -1, w, 1) + dss[id];
                        if (nstop < 1) nstop = 1;
                    }
                    nv = fwd_records(s, o, d, a0, a1, nstop, w, 1);
                    work_reserve(w, 1, nv + 1);
                    rev_sweep(s, w->buf[1], nv, g, NULL, w->dvs[1], NULL);
                }
                /* both lists are in ascending sample index: merge, missing = 0 */
                int64_t i = 0, j = 0;
                while (i < n || j < nv) {
                    int64_t ki = i < n ? w->buf[0][i].k : INT64_MAX;
                    int64_t kj = j < nv ? w->buf[1][j].k : INT64_MAX;
                    if (ki == kj) {
                        add_amb(amb, &w->buf[0][i], fabs(w->dvs[1][j] - w->dvs[0][i]));
                        ++i;
                        ++j;
                    } else if (ki < kj) {
                        add_amb(amb, &w->buf[0][i], fabs(w->dvs[0][i]));
                        ++i;
                    } else {
                        add_amb(amb, &w->buf[1][j], fabs(w->dvs[1][j]));
                        ++j;
                    }
                }
            }
}

typedef struct {
    const orc_scene* s;
    const orc_camera* cams;
    int32_t ncams;
    const double* dimg; /* ncams x H x W x 4 */
    int64_t next;
    pthread_mutex_t mu;
    /* per-thread accumulators, merged under the mutex at the end */
    double* dtf;   /* ntf x 4 */
    double* dvol;  /* nx*ny*nz or NULL */
    double* amb;   /* nx*ny*nz or NULL */
    int64_t total;
} grad_job;

static void* grad_worker(void* arg)
{
    grad_job* j = (grad_job*)arg;
    const orc_scene* s = j->s;
    int64_t nvox = s->nx * s->ny * s->nz;
    double* dtf = (double*)calloc((size_t)s->ntf * 4, sizeof(double));
    double* dvol = j->dvol ? (double*)calloc((size_t)nvox, sizeof(double)) : NULL;
    double* amb = j->amb ? (double*)calloc((size_t)nvox, sizeof(double)) : NULL;
    ray_work w;
    memset(&w, 0, sizeof(w));
    const int64_t chunk = 64;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i0 = j->next;
        j->next += chunk;
        pthread_mutex_unlock(&j->mu);
        if (i0 >= j->total) break;
        int64_t i1 = i0 + chunk < j->total ? i0 + chunk : j->total;
        for (int64_t i = i0; i < i1; ++i) {
            /* flat over (camera, py, px); all cameras have the same size */
            int64_t W = j->cams[0].width, H = j->cams[0].height;
            int64_t ci = i / (W * H), r = i % (W * H);
            const double* g = j->dimg + 4 * i;
            if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0 && g[3] == 0.0) continue;
            ray_backward(s, &j->cams[ci], r % W, r / W, g, dtf, dvol, amb, &w);
        }
    }
    pthread_mutex_lock(&j->mu);
    for (int64_t i = 0; i < (int64_t)s->ntf * 4; ++i) j->dtf[i] += dtf[i];
    if (dvol)
        for (int64_t i = 0; i < nvox; ++i) j->dvol[i] += dvol[i];
    if (amb)
        for (int64_t i = 0; i < nvox; ++i) j->amb[i] += amb[i];
    pthread_mutex_unlock(&j->mu);
    free(dtf);
    free(dvol);
    free(amb);
    for (int b = 0; b < 2; ++b) {
        free(w.buf[b]);
        free(w.dvs[b]);
    }
    free(w.alt);
    return NULL;
}

/*
 * Gradient of a loss with respect to the table (out_dtf, ntf x 4) and the
 * voxels (out_dvol, nx*ny*nz, may be NULL), given dL/dI (ncams x H x W x 4)
 * for the images of the composite (or MIP) renders of the cameras.  out_amb
 * (nx*ny*nz, may be NULL) receives the per-voxel bound of ray_backward on the
 * legitimate deviation of a renderer's voxel gradient.  All outputs are
 * overwritten.  Each thread holds its own voxel accumulators.
 */
int orc_backward(const orc_scene* s, const orc_camera* cams, int32_t ncams, const double* dimg,
                 double* out_dtf, double* out_dvol, double* out_amb, int nthreads)
{
    if (!scene_ok(s) || !cams || ncams <= 0 || !dimg || !out_dtf) return -1;
    for (int i = 1; i < ncams; ++i)
        if (cams[i].width != cams[0].width || cams[i].height != cams[0].height) return -1;
    int64_t nvox = s->nx * s->ny * s->nz;
    memset(out_dtf, 0, sizeof(double) * (size_t)s->ntf * 4);
    if (out_dvol) memset(out_dvol, 0, sizeof(double) * (size_t)nvox);
    if (out_amb) memset(out_amb, 0, sizeof(double) * (size_t)nvox);
    grad_job j;
    memset(&j, 0, sizeof(j));
    j.s = s;
    j.cams = cams;
    j.ncams = ncams;
    j.dimg = dimg;
    j.next = 0;
    pthread_mutex_init(&j.mu, NULL);
    j.dtf = out_dtf;
    j.dvol = out_dvol;
    j.amb = out_amb;
    j.total = (int64_t)ncams * cams[0].width * cams[0].height;
    run_threads(grad_worker, &j, nthreads);
    pthread_mutex_destroy(&j.mu);
    return 0;
}

/* ------------------------------------------------------ touched-voxel census */
typedef struct {
    const orc_scene* s;
    const orc_camera* cam;
    const int64_t* pix;
    int64_t npix;
    uint8_t* mask;
    int64_t next;
    pthread_mutex_t mu;
} touch_job;

static void* touch_worker(void* arg)
{
    touch_job* j = (touch_job*)arg;
    const orc_scene* s = j->s;
    const int64_t chunk = 64;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i0 = j->next;
        j->next += chunk;
        pthread_mutex_unlock(&j->mu);
        if (i0 >= j->npix) break;
        int64_t i1 = i0 + chunk < j->npix ? i0 + chunk : j->npix;
        for (int64_t i = i0; i < i1; ++i) {
            int64_t flat = j->pix ? j->pix[i] : i;
            int64_t px = flat % j->cam->width, py = flat / j->cam->width;
            double o[3], d[3];
            int64_t k0, k1;
            int flags = 0;
            camera_ray(j->cam, px, py, o, d);
            if (!ray_samples(s, o, d, &k0, &k1, &flags)) continue;
            double T = 1.0;
            for (int64_t k = k0; k < k1; ++k) {
                double t = (double)k * s->step;
                double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                int64_t idx[8];
                double w[8];
                double v = trilinear(s, p, idx, w, NULL);
                for (int c = 0; c < 8; ++c) __atomic_store_n(&j->mask[idx[c]], 1, __ATOMIC_RELAXED);
                if (s->mode == 0) {
                    tf_eval_t e;
                    tf_lookup(s, v, &e);
                    T *= (1.0 - e.rgba[3]);
                    if (s->ert <= 1.0 && 1.0 - T >= s->ert) break;
                }
            }
        }
    }
    return NULL;
}

/*
 * Mark in mask (nx*ny*nz bytes, caller-zeroed) every voxel that some executed
 * sample of the listed pixels reads (the 8 clamped trilinear corners).
 */
int orc_touch(const orc_scene* s, const orc_camera* cam, const int64_t* pix, int64_t npix,
              uint8_t* mask, int nthreads)
{
    if (!scene_ok(s) || !cam || !mask) return -1;
    if (!pix) npix = (int64_t)cam->width * cam->height;
    touch_job j = {s, cam, pix, npix, mask, 0, PTHREAD_MUTEX_INITIALIZER};
    run_threads(touch_worker, &j, nthreads);
    return 0;
}

/* Round float32 values to bfloat16 (round to nearest, ties to even), kept as float32. */
void orc_round_bf16(const float* in, float* out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], 4);
        if ((u & 0x7f800000u) == 0x7f800000u) {
            /* inf / nan: keep (quiet the nan) */
            if (u & 0x007fffffu) u |= 0x00400000u;
            u &= 0xffff0000u;
        } else {
            uint32_t lsb = (u >> 16) & 1u;
            u = (u + 0x7fffu + lsb) & 0xffff0000u;
        }
        memcpy(&out[i], &u, 4);
    }
}

/* ------------------------------------------------------------ image pyramid */
/*
 * Levels of a premultiplied RGBA image for viewers that show a high-resolution
 * render at several zoom levels (Sec. 3: static renders of one orientation at
 * user-chosen sizes, cut into tiles for display).  Level 0 is the image,
 * W x H; level l+1 is ceil(W_l / 2) x ceil(H_l / 2), and its pixel (x, y) is
 * the mean of the pixels (2x + i, 2y + j), i, j in {0, 1}, of level l that lie
 * inside level l (one, two or four of them).  Premultiplied colour makes this
 * box filter the right one for alpha.
 *
 * Output: levels 1 .. L-1 (L = number of levels down to 1 x 1, counting level
 * 0) one after the other, 4 doubles a pixel, each level either row-major
 * (tile = 0) or as ceil(W/tile) x ceil(H/tile) tiles of tile x tile pixels,
 * tiles row-major, pixels row-major inside a tile, with zeros where a tile
 * passes the level's edge.  Returns the number of levels L, or -1 on bad
 * arguments.  out may be NULL to size it: *nout receives the doubles needed.
 */
static int64_t pyr_level_pixels(int64_t w, int64_t h, int64_t tile)
{
    if (tile <= 0) return w * h;
    int64_t tx = (w + tile - 1) / tile, ty = (h + tile - 1) / tile;
    return tx * ty * tile * tile;
}

static int64_t pyr_index(int64_t x, int64_t y, int64_t w, int64_t tile)
{
    if (tile <= 0) return y * w + x;
    int64_t tx = (w + tile - 1) / tile;
    return ((y / tile) * tx + x / tile) * tile * tile + (y % tile) * tile + (x % tile);
}

int orc_pyramid(const float* img, int64_t w, int64_t h, int64_t tile, double* out, int64_t* nout)
{
    if (w <= 0 || h <= 0 || tile < 0) return -1;
    int levels = 1;
    int64_t total = 0;
    for (int64_t lw = w, lh = h; lw > 1 || lh > 1;) {
        lw = (lw + 1) / 2;
        lh = (lh + 1) / 2;
        total += 4 * pyr_level_pixels(lw, lh, tile);
        ++levels;
    }
    if (nout) *nout = total;
    if (!out) return levels;
    memset(out, 0, sizeof(double) * (size_t)total);
    /* the previous level, row-major, in double */
    double* prev = (double*)malloc(sizeof(double) * 4 * (size_t)(w * h));
    for (int64_t i = 0; i < 4 * w * h; ++i) prev[i] = (double)img[i];
    int64_t pw = w, ph = h, off = 0;
    while (pw > 1 || ph > 1) {
        int64_t lw = (pw + 1) / 2, lh = (ph + 1) / 2;
        double* cur = (double*)malloc(sizeof(double) * 4 * (size_t)(lw * lh));
        for (int64_t y = 0; y < lh; ++y)
            for (int64_t x = 0; x < lw; ++x) {
                double acc[4] = {0, 0, 0, 0};
                int n = 0;
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) {
                        int64_t sx = 2 * x + i, sy = 2 * y + j;
                        if (sx >= pw || sy >= ph) continue;
                        for (int c = 0; c < 4; ++c) acc[c] += prev[4 * (sy * pw + sx) + c];
                        ++n;
                    }
                for (int c = 0; c < 4; ++c) {
                    cur[4 * (y * lw + x) + c] = acc[c] / (double)n;
                    out[off + 4 * pyr_index(x, y, lw, tile) + c] = acc[c] / (double)n;
                }
            }
        off += 4 * pyr_level_pixels(lw, lh, tile);
        free(prev);
        prev = cur;
        pw = lw;
        ph = lh;
    }
    free(prev);
    return levels;
}

/* -------------------------------------------------------- catalogue overlay */
/*
 * Wireframe bounding cubes of a source catalogue over a render (Sec. 2: a
 * source finder's detections, given as bounding cubes, are superimposed as
 * wireframe boxes on the volume rendering, one colour per catalogue).
 *
 * Each of the 12 edges of a box is projected through the camera's inverse
 * mapping: for the basis M = [right | up | fwd] (columns) and q = p - eye,
 * (a, b, c) = M^-1 q; a perspective camera gives window coordinates
 * (u, v) = (a / c, b / c) (the part of an edge with c < 1e-3 is clipped
 * away), an orthographic one (u, v) = (a, b).  Continuous pixel coordinates
 * are X = (u - l) W / (r - l) - 1/2, Y = (t - v) H / (t - b) - 1/2 (pixel
 * centres at integers).  The 2-D segment is clipped to [-1, W] x [-1, H]
 * (Liang-Barsky) and walked with n + 1 evenly spaced points, n =
 * max(1, ceil(max(|dX|, |dY|))), each marking pixel (floor(X + 1/2),
 * floor(Y + 1/2)) when it lies in the image.  A pixel keeps the highest box
 * index that marks it; its premultiplied colour C, alpha A then become
 * a c + (1 - a) C, a + (1 - a) A with the box's straight colour (c, a).
 * All arithmetic is double precision, one rounding per operation, in the
 * order written here.
 */
static void basis_inverse(const double R[3], const double U[3], const double F[3], double inv[9])
{
    /* m[i][j]: column 0 = right, 1 = up, 2 = fwd */
    double m00 = R[0], m01 = U[0], m02 = F[0];
    double m10 = R[1], m11 = U[1], m12 = F[1];
    double m20 = R[2], m21 = U[2], m22 = F[2];
    double c0 = m11 * m22 - m12 * m21;
    double c1 = m12 * m20 - m10 * m22;
    double c2 = m10 * m21 - m11 * m20;
    double det = m00 * c0 + m01 * c1 + m02 * c2;
    inv[0] = c0 / det;
    inv[1] = (m02 * m21 - m01 * m22) / det;
    inv[2] = (m01 * m12 - m02 * m11) / det;
    inv[3] = c1 / det;
    inv[4] = (m00 * m22 - m02 * m20) / det;
    inv[5] = (m02 * m10 - m00 * m12) / det;
    inv[6] = c2 / det;
    inv[7] = (m01 * m20 - m00 * m21) / det;
    inv[8] = (m00 * m11 - m01 * m10) / det;
}

static void cam_coords(const double inv[9], const double eye[3], const double p[3], double out[3])
{
    double q0 = p[0] - eye[0], q1 = p[1] - eye[1], q2 = p[2] - eye[2];
    out[0] = inv[0] * q0 + inv[1] * q1 + inv[2] * q2;
    out[1] = inv[3] * q0 + inv[4] * q1 + inv[5] * q2;
    out[2] = inv[6] * q0 + inv[7] * q1 + inv[8] * q2;
}

/* Liang-Barsky: clip s in [*s0, *s1] of x0 + s dx to lo <= x <= hi; 0 if empty */
static int clip_axis(double x0, double dx, double lo, double hi, double* s0, double* s1)
{
    if (dx == 0.0) return (x0 >= lo && x0 <= hi);
    double a = (lo - x0) / dx, b = (hi - x0) / dx;
    if (a > b) {
        double t = a;
        a = b;
        b = t;
    }
    if (a > *s0) *s0 = a;
    if (b < *s1) *s1 = b;
    return *s0 <= *s1;
}

int orc_overlay(const orc_camera* cam, const double* boxes, int64_t nbox, const float* colours,
                double* img, int32_t* key)
{
    if (!cam || (nbox > 0 && (!boxes || !colours)) || !img || !key) return -1;
    const int64_t W = cam->width, H = cam->height;
    double inv[9];
    basis_inverse(cam->right, cam->up, cam->fwd, inv);
    const double l = cam->win[0], r = cam->win[1], b = cam->win[2], t = cam->win[3];
    const double sx = (double)W / (r - l), sy = (double)H / (t - b);
    memset(key, 0, sizeof(int32_t) * (size_t)(W * H));
    for (int64_t bi = 0; bi < nbox; ++bi) {
        const double* bx = boxes + 6 * bi;
        for (int e = 0; e < 12; ++e) {
            int axis = e / 4, rest = e % 4;
            double p0[3], p1[3];
            int o = 0;
            for (int a = 0; a < 3; ++a) {
                if (a == axis) {
                    p0[a] = bx[a];
                    p1[a] = bx[3 + a];
                } else {
                    int bit = (rest >> o) & 1;
                    ++o;
                    p0[a] = p1[a] = bit ? bx[3 + a] : bx[a];
                }
            }
            double c0[3], c1[3];
            cam_coords(inv, cam->eye, p0, c0);
            cam_coords(inv, cam->eye, p1, c1);
            double u0, v0, u1, v1;
            if (cam->type == 1) {
                const double nearc = 1e-3;
                if (c0[2] < nearc && c1[2] < nearc) continue;
                if (c0[2] < nearc || c1[2] < nearc) {
                    double s = (nearc - c0[2]) / (c1[2] - c0[2]);
                    double* lo = c0[2] < nearc ? c0 : c1;
                    double m0 = c0[0] + s * (c1[0] - c0[0]);
                    double m1 = c0[1] + s * (c1[1] - c0[1]);
                    lo[0] = m0;
                    lo[1] = m1;
                    lo[2] = nearc;
                }
                u0 = c0[0] / c0[2];
                v0 = c0[1] / c0[2];
                u1 = c1[0] / c1[2];
                v1 = c1[1] / c1[2];
            } else {
                u0 = c0[0];
                v0 = c0[1];
                u1 = c1[0];
                v1 = c1[1];
            }
            double X0 = (u0 - l) * sx - 0.5, Y0 = (t - v0) * sy - 0.5;
            double X1 = (u1 - l) * sx - 0.5, Y1 = (t - v1) * sy - 0.5;
            double dX = X1 - X0, dY = Y1 - Y0, s0 = 0.0, s1 = 1.0;
            if (!clip_axis(X0, dX, -1.0, (double)W, &s0, &s1)) continue;
            if (!clip_axis(Y0, dY, -1.0, (double)H, &s0, &s1)) continue;
            double A0 = X0 + s0 * dX, B0 = Y0 + s0 * dY;
            double A1 = X0 + s1 * dX, B1 = Y0 + s1 * dY;
            double dA = A1 - A0, dB = B1 - B0;
            double len = fabs(dA) > fabs(dB) ? fabs(dA) : fabs(dB);
            int64_t n = (int64_t)ceil(len);
            if (n < 1) n = 1;
            for (int64_t i = 0; i <= n; ++i) {
                double f = (double)i / (double)n;
                int64_t px = (int64_t)floor(A0 + dA * f + 0.5);
                int64_t py = (int64_t)floor(B0 + dB * f + 0.5);
                if (px < 0 || px >= W || py < 0 || py >= H) continue;
                int32_t k = (int32_t)(bi + 1);
                if (key[py * W + px] < k) key[py * W + px] = k;
            }
        }
    }
    for (int64_t i = 0; i < W * H; ++i) {
        if (!key[i]) continue;
        const float* c = colours + 4 * (key[i] - 1);
        double a = (double)c[3];
        for (int ch = 0; ch < 3; ++ch) img[4 * i + ch] = a * (double)c[ch] + (1.0 - a) * img[4 * i + ch];
        img[4 * i + 3] = a + (1.0 - a) * img[4 * i + 3];
    }
    return 0;
}
