/*
 * dpv_oracle.c -- plain, slow, FP64 CPU oracle for the data-parallel volume
 * rendering path (sort-last compositing of per-brick ray-march fragments).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it follows (arXiv 2407.00179, "Standardized Data-Parallel Rendering
 * Using ANARI"):
 *   - each rank owns one spatial part of a jointly defined world (§1, §3.1.2);
 *   - ghost layers make local effects correct across part borders (§1);
 *   - each rank reduces its render to one fragment (colour, opacity, depth)
 *     per pixel, which is correct for convex parts (§2.1);
 *   - fragments carry RGBA and depth and are sorted per pixel, then blended
 *     front to back (§5.1.1, "Compositing");
 *   - the final frame exists on rank 0 (§3.1.3).
 * The paper gives no rendering equations.  The emission-absorption model,
 * the sampling rule and everything numeric are readings of that text,
 * each stated where it is used.
 *
 * Everything is FP64.  Stored brick values (f32, f16, bf16, fp8 e4m3) are
 * decoded per access and never copied into an FP64 array.
 *
 * Parity status: every function below is pinned by a CPU test against a
 * closed form, an invariant, a library routine or brute force.  The camera
 * convention (the paper fixes none) is pinned by geometric properties and
 * by the OpenGL look-at / perspective unprojection of each pixel centre.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_F32 0
#define ORC_F16 1
#define ORC_BF16 2
#define ORC_FP8 3

#define ORC_KEY_EMPTY 2147483647

#define ORC_FLAG_HIT 1
#define ORC_FLAG_EXIT_AMBIG 2
#define ORC_FLAG_OWNER_AMBIG 4
#define ORC_FLAG_ERT_AMBIG 8
#define ORC_FLAG_ISO_AMBIG 16

typedef struct {
    int dims[3];          /* nodes per axis */
    double origin[3];     /* world position of node (0,0,0) */
    double spacing;       /* world distance between nodes */
} orc_grid;

typedef struct {
    double eye[3], center[3], up[3];
    double fovy_deg;
} orc_camera;

typedef struct {
    int width, height;
    double step_voxels;   /* dt = step_voxels * spacing (world units) */
    double sigma_max;     /* extinction per world unit at TF alpha 1 */
    double ert;           /* per-fragment early termination; <=0 or >=1: off */
    double amb_samples;   /* ambiguity band, in samples, for flags */
    double amb_alpha;     /* ambiguity band on opacity, for ERT flags */
} orc_frame;

typedef struct {
    int owned_lo[3], owned_hi[3];   /* half-open node range owned */
    int dtype;                      /* ORC_F32 .. ORC_FP8 */
    double scale;                   /* value = scale * stored */
    const void* data;               /* stored nodes (see orc_stored_box), x fastest */
} orc_brick;

typedef struct {
    const float* rgba;    /* n x 4 */
    int n;
    double vmin, vmax;
} orc_tf;

/* ------------------------------------------------------------------------ */
/* number formats                                                            */
/* ------------------------------------------------------------------------ */

/* IEEE binary16 -> double. */
static double dec_f16(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1.0 + m / 1024.0, e - 15);
    return s ? -v : v;
}

/* bfloat16 (upper half of a binary32) -> double. */
static double dec_bf16(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* OCP FP8 E4M3 ("fn": no infinities, S.1111.111 is NaN, max 448) -> double. */
static double dec_fp8(uint8_t b) {
    int s = (b >> 7) & 1, e = (b >> 3) & 15, m = b & 7;
    double v;
    if (e == 0) v = ldexp((double)m, -9);
    else if (e == 15 && m == 7) v = NAN;
    else v = ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

static double decode(const void* data, int dtype, int64_t i) {
    switch (dtype) {
        case ORC_F32: return (double)((const float*)data)[i];
        case ORC_F16: return dec_f16(((const uint16_t*)data)[i]);
        case ORC_BF16: return dec_bf16(((const uint16_t*)data)[i]);
        default: return dec_fp8(((const uint8_t*)data)[i]);
    }
}

/* Round x to the nearest value with `mbits` fraction bits, exponent >= emin
 * (subnormals below), ties to even.  Overflow beyond maxv gives +-inf, or
 * +-maxv when `sat`. */
static double round_format(double x, int mbits, int emin, double maxv, int sat) {
    if (x == 0.0 || isnan(x)) return x;
    double a = fabs(x);
    int E;
    frexp(a, &E);                      /* a = f * 2^E, f in [0.5, 1) */
    int e = E - 1;                     /* exponent of the leading bit */
    if (e < emin) e = emin;
    double q = ldexp(1.0, e - mbits);  /* spacing of representable values */
    double r = nearbyint(a / q) * q;   /* a / q is exact; nearbyint ties to even */
    if (r > maxv) r = sat ? maxv : INFINITY;
    return copysign(r, x);
}

static uint16_t enc_f16(float f) {
    double r = round_format((double)f, 10, -14, 65504.0, 0);
    uint16_t s = signbit(r) ? 0x8000 : 0;
    double a = fabs(r);
    if (isinf(a)) return s | 0x7C00;
    if (a == 0.0) return s;
    int E;
    frexp(a, &E);
    int e = E - 1;
    if (e < -14) return s | (uint16_t)(a / ldexp(1.0, -24));        /* subnormal */
    return s | (uint16_t)((e + 15) << 10) | (uint16_t)((a / ldexp(1.0, e) - 1.0) * 1024.0);
}

static uint16_t enc_bf16(float f) {
    double r = round_format((double)f, 7, -126, 3.3895313892515355e38, 0);
    float g = (float)r;
    uint32_t u;
    memcpy(&u, &g, 4);
    return (uint16_t)(u >> 16);
}

static uint8_t enc_fp8(float f) {
    double r = round_format((double)f, 3, -6, 448.0, 1);   /* saturating */
    uint8_t s = signbit(r) ? 0x80 : 0;
    double a = fabs(r);
    if (a == 0.0) return s;
    int E;
    frexp(a, &E);
    int e = E - 1;
    if (e < -6) return s | (uint8_t)(a / ldexp(1.0, -9));
    return s | (uint8_t)((e + 7) << 3) | (uint8_t)((a / ldexp(1.0, e) - 1.0) * 8.0);
}

/* Per-brick scale for a storage format: fp8 maps max|v| of the brick's stored
 * nodes onto 448 (computed in float32: max|v| / 448); the others use 1. */
float orc_brick_scale(const float* v, int64_t n, int dtype) {
    if (dtype != ORC_FP8) return 1.0f;
    float m = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        float a = fabsf(v[i]);
        if (a > m) m = a;
    }
    return m > 0.0f ? m / 448.0f : 1.0f;
}

/* Quantise float32 values to a storage format: stored = round(v / scale),
 * the division in float32, rounding to nearest even (fp8 saturates). */
void orc_quantize(const float* v, int64_t n, int dtype, float scale, void* out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float q = v[i] / scale;
        switch (dtype) {
            case ORC_F32: ((float*)out)[i] = q; break;
            case ORC_F16: ((uint16_t*)out)[i] = enc_f16(q); break;
            case ORC_BF16: ((uint16_t*)out)[i] = enc_bf16(q); break;
            default: ((uint8_t*)out)[i] = enc_fp8(q); break;
        }
    }
}

void orc_dequantize(const void* data, int64_t n, int dtype, double scale, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = scale * decode(data, dtype, i);
}

/* ------------------------------------------------------------------------ */
/* bricks                                                                    */
/* ------------------------------------------------------------------------ */

/* Nodes a rank stores: its owned nodes [lo, hi) plus one ghost node on each
 * side, clipped to the volume.  Writes first node and node count per axis. */
void orc_stored_box(const int dims[3], const int lo[3], const int hi[3], int s_lo[3], int s_n[3]) {
    for (int a = 0; a < 3; ++a) {
        int l = lo[a] - 1 < 0 ? 0 : lo[a] - 1;
        int h = hi[a] > dims[a] - 1 ? dims[a] - 1 : hi[a];
        s_lo[a] = l;
        s_n[a] = h - l + 1;
    }
}

/* Copy a brick's stored nodes out of the global float32 field (x fastest). */
void orc_extract_brick(const float* field, const int dims[3], const int lo[3], const int hi[3], float* out) {
    int s_lo[3], s_n[3];
    orc_stored_box(dims, lo, hi, s_lo, s_n);
    int64_t k = 0;
    for (int z = 0; z < s_n[2]; ++z)
        for (int y = 0; y < s_n[1]; ++y)
            for (int x = 0; x < s_n[0]; ++x)
                out[k++] = field[((int64_t)(z + s_lo[2]) * dims[1] + (y + s_lo[1])) * dims[0] + (x + s_lo[0])];
}

/* Owned region of a brick in node coordinates: [lo - 1/2, hi - 1/2] per axis,
 * clipped to the volume box [0, n - 1]. */
static void owned_region(const orc_grid* g, const orc_brick* b, double r0[3], double r1[3]) {
    for (int a = 0; a < 3; ++a) {
        double l = b->owned_lo[a] - 0.5, h = b->owned_hi[a] - 0.5;
        r0[a] = l < 0.0 ? 0.0 : l;
        r1[a] = h > g->dims[a] - 1 ? g->dims[a] - 1 : h;
    }
}

/* Does node-space point q lie in the brick's owned region?  Half-open
 * [r0, r1) per axis, except that the volume's upper face is closed. */
static int owns(const orc_grid* g, const orc_brick* b, const double q[3]) {
    double r0[3], r1[3];
    owned_region(g, b, r0, r1);
    for (int a = 0; a < 3; ++a) {
        if (q[a] < r0[a]) return 0;
        if (b->owned_hi[a] >= g->dims[a]) {
            if (q[a] > r1[a]) return 0;
        } else if (q[a] >= r1[a]) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* trilinear interpolation                                                   */
/* ------------------------------------------------------------------------ */

/* Trilinear value at node-space point q from a box of nodes [b_lo, b_lo+b_n)
 * stored x fastest.  Cell index i = clamp(floor(q), b_lo, b_lo + b_n - 2),
 * weights f = q - i, then lerp in x, y, z.  Corner values are decoded (and
 * scaled) before interpolation.  Optionally returns the 8 corner indices
 * (into the box) and weights, corner c = dx + 2 dy + 4 dz. */
static double trilinear(const void* data, int dtype, double scale, const int b_lo[3], const int b_n[3],
                        const double q[3], int64_t idx[8], double w[8]) {
    int i[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        int c = (int)floor(q[a]);
        if (c < b_lo[a]) c = b_lo[a];
        if (c > b_lo[a] + b_n[a] - 2) c = b_lo[a] + b_n[a] - 2;
        i[a] = c - b_lo[a];
        f[a] = q[a] - c;
    }
    double v[8];
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        int64_t k = ((int64_t)(i[2] + dz) * b_n[1] + (i[1] + dy)) * b_n[0] + (i[0] + dx);
        v[c] = scale * decode(data, dtype, k);
        if (idx) idx[c] = k;
        if (w) w[c] = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
    }
    double x00 = v[0] + f[0] * (v[1] - v[0]);
    double x10 = v[2] + f[0] * (v[3] - v[2]);
    double x01 = v[4] + f[0] * (v[5] - v[4]);
    double x11 = v[6] + f[0] * (v[7] - v[6]);
    double y0 = x00 + f[1] * (x10 - x00);
    double y1 = x01 + f[1] * (x11 - x01);
    return y0 + f[2] * (y1 - y0);
}

/* ------------------------------------------------------------------------ */
/* transfer function                                                         */
/* ------------------------------------------------------------------------ */

/* Piecewise-linear RGBA lookup: u = clamp((s - vmin) / (vmax - vmin), 0, 1) *
 * (N - 1), i0 = min(floor(u), N - 2), w = u - i0, value = (1 - w) Tab[i0] +
 * w Tab[i0 + 1].  Also returns i0, w and du/ds (0 where clamped). */
static void tf_lookup(const orc_tf* tf, double s, double out[4], int* i0_out, double* w_out, double* duds) {
    double x = (s - tf->vmin) / (tf->vmax - tf->vmin);
    double d = (double)(tf->n - 1) / (tf->vmax - tf->vmin);
    if (x < 0.0) { x = 0.0; d = 0.0; }
    if (x > 1.0) { x = 1.0; d = 0.0; }
    double u = x * (tf->n - 1);
    int i0 = (int)floor(u);
    if (i0 > tf->n - 2) i0 = tf->n - 2;
    double w = u - i0;
    for (int c = 0; c < 4; ++c)
        out[c] = (1.0 - w) * tf->rgba[4 * i0 + c] + w * tf->rgba[4 * (i0 + 1) + c];
    if (i0_out) *i0_out = i0;
    if (w_out) *w_out = w;
    if (duds) *duds = d;
}

/* ------------------------------------------------------------------------ */
/* camera                                                                    */
/* ------------------------------------------------------------------------ */

static void normalize3(double v[3]) {
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
}

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Pinhole camera, right-handed look-at: forward f = normalize(center - eye),
 * right r = normalize(f x up), true up u = r x f.  Pixel (px, py), row 0 at
 * the bottom, is hit through its centre: ndc = ((px + 1/2) / W * 2 - 1) * W/H
 * horizontally and (py + 1/2) / H * 2 - 1 vertically; the direction is
 * normalize(f + ndc_x tan(fovy/2) r + ndc_y tan(fovy/2) u), origin the eye. */
void orc_camera_ray(const orc_camera* c, int W, int H, int px, int py, double o[3], double d[3]) {
    double f[3] = {c->center[0] - c->eye[0], c->center[1] - c->eye[1], c->center[2] - c->eye[2]};
    normalize3(f);
    double r[3], u[3];
    cross3(f, c->up, r);
    normalize3(r);
    cross3(r, f, u);
    double th = tan(c->fovy_deg * M_PI / 360.0);
    double nx = (((px + 0.5) / W) * 2.0 - 1.0) * ((double)W / H);
    double ny = ((py + 0.5) / H) * 2.0 - 1.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = f[a] + nx * th * r[a] + ny * th * u[a];
        o[a] = c->eye[a];
    }
    normalize3(d);
}

/* Ray against the axis-aligned world box [lo, hi]: parametric interval,
 * clipped to t >= 0.  Returns 1 when non-empty. */
static int ray_box(const double o[3], const double d[3], const double lo[3], const double hi[3],
                   double* t0, double* t1) {
    double a = 0.0, b = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < lo[k] || o[k] > hi[k]) return 0;
            continue;
        }
        double ta = (lo[k] - o[k]) / d[k], tb = (hi[k] - o[k]) / d[k];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > a) a = ta;
        if (tb < b) b = tb;
    }
    *t0 = a;
    *t1 = b;
    return a < b;
}

/* ------------------------------------------------------------------------ */
/* samples along a ray                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double o[3], d[3];
    double t_enter, t_exit, dt;
    int64_t n;            /* number of samples */
    int flags;
} orc_rayinfo;

/* Ray of pixel (px, py) against the whole volume box; samples sit at
 * t_j = t_enter + (j + 1/2) dt for every j >= 0 with t_j < t_exit. */
static void ray_samples(const orc_grid* g, const orc_camera* cam, const orc_frame* fr, int px, int py,
                        orc_rayinfo* ri) {
    orc_camera_ray(cam, fr->width, fr->height, px, py, ri->o, ri->d);
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = g->origin[a];
        hi[a] = g->origin[a] + (g->dims[a] - 1) * g->spacing;
    }
    ri->dt = fr->step_voxels * g->spacing;
    ri->n = 0;
    ri->flags = 0;
    if (!ray_box(ri->o, ri->d, lo, hi, &ri->t_enter, &ri->t_exit)) return;
    ri->flags |= ORC_FLAG_HIT;
    double x = (ri->t_exit - ri->t_enter) / ri->dt - 0.5;
    int64_t n = (int64_t)ceil(x);
    if (n < 0) n = 0;
    while (n > 0 && ri->t_enter + (n - 0.5) * ri->dt >= ri->t_exit) --n;
    while (ri->t_enter + (n + 0.5) * ri->dt < ri->t_exit) ++n;
    ri->n = n;
    if (fabs(x - nearbyint(x)) < fr->amb_samples) ri->flags |= ORC_FLAG_EXIT_AMBIG;
}

static void sample_point(const orc_grid* g, const orc_rayinfo* ri, int64_t j, double q[3], double* t) {
    double tj = ri->t_enter + (j + 0.5) * ri->dt;
    for (int a = 0; a < 3; ++a) {
        double p = ri->o[a] + tj * ri->d[a];
        q[a] = (p - g->origin[a]) / g->spacing;
        if (q[a] < 0.0) q[a] = 0.0;                       /* rounding at the box */
        if (q[a] > g->dims[a] - 1) q[a] = g->dims[a] - 1;
    }
    if (t) *t = tj;
}

/* ------------------------------------------------------------------------ */
/* emission-absorption                                                       */
/* ------------------------------------------------------------------------ */

/* Classify one sample: TF colour c and opacity alpha = 1 - exp(-sigma dt)
 * with sigma = sigma_max * a. */
static void classify(const orc_tf* tf, const orc_frame* fr, double dt, double s, double c[3], double* alpha) {
    double v[4];
    tf_lookup(tf, s, v, NULL, NULL, NULL);
    c[0] = v[0]; c[1] = v[1]; c[2] = v[2];
    *alpha = 1.0 - exp(-fr->sigma_max * v[3] * dt);
}

/* Unpartitioned render of the global float32 field: front-to-back
 * C += T alpha c, T *= (1 - alpha), A = 1 - T over every sample of the ray,
 * no early termination.  This is the plain definition every partitioned
 * result must reproduce.  Outputs per listed pixel: rgba (premultiplied),
 * sample count, flags. */
void orc_render_full(const orc_grid* g, const float* field, const orc_tf* tf, const orc_camera* cam,
                     const orc_frame* fr, int npix, const int32_t* pix,
                     double* rgba, int64_t* nsamples, uint8_t* flags) {
    int all_lo[3] = {0, 0, 0};
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < npix; ++k) {
        int p = pix ? pix[k] : k;
        orc_rayinfo ri;
        ray_samples(g, cam, fr, p % fr->width, p / fr->width, &ri);
        double C[3] = {0, 0, 0}, T = 1.0;
        for (int64_t j = 0; j < ri.n; ++j) {
            double q[3];
            sample_point(g, &ri, j, q, NULL);
            double s = trilinear(field, ORC_F32, 1.0, all_lo, g->dims, q, NULL, NULL);
            double c[3], al;
            classify(tf, fr, ri.dt, s, c, &al);
            for (int a = 0; a < 3; ++a) C[a] += T * al * c[a];
            T *= 1.0 - al;
        }
        rgba[4 * k + 0] = C[0];
        rgba[4 * k + 1] = C[1];
        rgba[4 * k + 2] = C[2];
        rgba[4 * k + 3] = 1.0 - T;
        if (nsamples) nsamples[k] = ri.n;
        if (flags) flags[k] = (uint8_t)ri.flags;
    }
}

/* ------------------------------------------------------------------------ */
/* per-brick fragments and sort-last compositing                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double C[3], T;
    int64_t key;          /* first global sample index, or EMPTY */
    int32_t nsamp;        /* samples evaluated */
    int done;             /* early-terminated */
    double margin;        /* distance of opacity to the ERT threshold at stop */
} frag_state;

static int find_owner(const orc_grid* g, int K, const orc_brick* b, const double q[3], int hint) {
    if (hint >= 0 && owns(g, &b[hint], q)) return hint;
    for (int k = 0; k < K; ++k)
        if (owns(g, &b[k], q)) return k;
    return -1;
}

/* Is the sample within `band` samples of an internal face of its owner? */
static int near_internal_face(const orc_grid* g, const orc_brick* b, const orc_rayinfo* ri, double tj,
                              double band) {
    double r0[3], r1[3];
    owned_region(g, b, r0, r1);
    for (int a = 0; a < 3; ++a) {
        if (ri->d[a] == 0.0) continue;
        double faces[2] = {r0[a], r1[a]};
        int internal[2] = {b->owned_lo[a] > 0, b->owned_hi[a] < g->dims[a]};
        for (int s = 0; s < 2; ++s) {
            if (!internal[s]) continue;
            double pw = g->origin[a] + faces[s] * g->spacing;
            double tf = (pw - ri->o[a]) / ri->d[a];
            if (fabs(tj - tf) < band * ri->dt) return 1;
        }
    }
    return 0;
}

/* Fragments of one pixel: every sample goes to the brick owning its
 * position; each brick front-to-back accumulates its own samples (with
 * per-fragment early termination when enabled).  Fragment = premultiplied
 * RGBA, key = global index of its first sample. */
static void pixel_fragments(const orc_grid* g, int K, const orc_brick* b, const orc_tf* tf,
                            const orc_frame* fr, const orc_rayinfo* ri, frag_state* fs, int* flags) {
    int bl[3], bn[3];
    for (int k = 0; k < K; ++k) {
        fs[k].C[0] = fs[k].C[1] = fs[k].C[2] = 0.0;
        fs[k].T = 1.0;
        fs[k].key = ORC_KEY_EMPTY;
        fs[k].nsamp = 0;
        fs[k].done = 0;
        fs[k].margin = INFINITY;
    }
    int ert_on = fr->ert > 0.0 && fr->ert < 1.0;
    int owner = -1;
    for (int64_t j = 0; j < ri->n; ++j) {
        double q[3], tj;
        sample_point(g, ri, j, q, &tj);
        owner = find_owner(g, K, b, q, owner);
        if (owner < 0) continue;     /* unreachable for a valid partition */
        frag_state* f = &fs[owner];
        if (near_internal_face(g, &b[owner], ri, tj, fr->amb_samples)) *flags |= ORC_FLAG_OWNER_AMBIG;
        if (f->key == ORC_KEY_EMPTY) f->key = j;
        if (f->done) continue;
        orc_stored_box(g->dims, b[owner].owned_lo, b[owner].owned_hi, bl, bn);
        double s = trilinear(b[owner].data, b[owner].dtype, b[owner].scale, bl, bn, q, NULL, NULL);
        double c[3], al;
        classify(tf, fr, ri->dt, s, c, &al);
        double A_before = 1.0 - f->T;
        for (int a = 0; a < 3; ++a) f->C[a] += f->T * al * c[a];
        f->T *= 1.0 - al;
        f->nsamp++;
        if (ert_on && 1.0 - f->T > fr->ert) {
            f->done = 1;
            double m1 = (1.0 - f->T) - fr->ert, m0 = fr->ert - A_before;
            f->margin = m1 < m0 ? m1 : m0;
            if (f->margin < fr->amb_alpha) *flags |= ORC_FLAG_ERT_AMBIG;
        }
    }
}

/* Order of a pixel's fragments: non-empty fragments by ascending key (keys
 * of non-empty fragments are distinct), written as brick ids, then 0xFF. */
static int fragment_order(int K, const frag_state* fs, uint8_t* order) {
    int m = 0;
    for (int k = 0; k < K; ++k)
        if (fs[k].key != ORC_KEY_EMPTY) order[m++] = (uint8_t)k;
    for (int i = 1; i < m; ++i) {          /* insertion sort by key */
        uint8_t v = order[i];
        int j = i - 1;
        while (j >= 0 && fs[order[j]].key > fs[v].key) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    for (int k = m; k < K; ++k) order[k] = 0xFF;
    return m;
}

/* Sort-last composite of one pixel: front-to-back "over" on premultiplied
 * RGBA, C += (1 - A) C_k, A += (1 - A) A_k, in key order.  Depth = t of the
 * first sample of the first fragment with A_k > 0, +inf if none. */
static void composite_pixel(int K, const frag_state* fs, const orc_rayinfo* ri, const uint8_t* order, int m,
                            double out[4], double* depth) {
    double C[3] = {0, 0, 0}, A = 0.0;
    *depth = INFINITY;
    for (int i = 0; i < m; ++i) {
        const frag_state* f = &fs[order[i]];
        double Ak = 1.0 - f->T;
        for (int a = 0; a < 3; ++a) C[a] += (1.0 - A) * f->C[a];
        A += (1.0 - A) * Ak;
        if (Ak > 0.0 && isinf(*depth)) *depth = ri->t_enter + (f->key + 0.5) * ri->dt;
    }
    (void)K;
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = A;
}

/* Partitioned render: fragments per brick, then sort-last composite.
 * Outputs per listed pixel k (any pointer may be NULL):
 *   rgba[4k..], depth[k]           composited frame
 *   order[K k ..]                  brick ids front to back, 0xFF padded
 *   frag_rgba[4 (K k + b) ..]      fragment of brick b (premultiplied)
 *   frag_key[K k + b]              first sample index or 2^31 - 1
 *   frag_nsamp[K k + b]            samples evaluated
 *   frag_margin[K k + b]           ERT margin (+inf if no stop)
 *   nsamples[k]                    samples evaluated, all bricks
 *   flags[k]                       ORC_FLAG_* bits */
void orc_render_bricks(const orc_grid* g, int K, const orc_brick* bricks, const orc_tf* tf,
                       const orc_camera* cam, const orc_frame* fr, int npix, const int32_t* pix,
                       double* rgba, double* depth, uint8_t* order, double* frag_rgba, int32_t* frag_key,
                       int32_t* frag_nsamp, double* frag_margin, int64_t* nsamples, uint8_t* flags) {
#pragma omp parallel
    {
        frag_state* fs = (frag_state*)malloc(sizeof(frag_state) * K);
        uint8_t* ord = (uint8_t*)malloc(K);
#pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < npix; ++k) {
            int p = pix ? pix[k] : k;
            orc_rayinfo ri;
            ray_samples(g, cam, fr, p % fr->width, p / fr->width, &ri);
            int fl = ri.flags;
            pixel_fragments(g, K, bricks, tf, fr, &ri, fs, &fl);
            int m = fragment_order(K, fs, ord);
            double out[4], dep;
            composite_pixel(K, fs, &ri, ord, m, out, &dep);
            if (rgba) for (int c = 0; c < 4; ++c) rgba[4 * k + c] = out[c];
            if (depth) depth[k] = dep;
            if (order) memcpy(order + (int64_t)K * k, ord, K);
            int64_t ns = 0;
            for (int b = 0; b < K; ++b) {
                int64_t o = (int64_t)K * k + b;
                if (frag_rgba) {
                    frag_rgba[4 * o + 0] = fs[b].C[0];
                    frag_rgba[4 * o + 1] = fs[b].C[1];
                    frag_rgba[4 * o + 2] = fs[b].C[2];
                    frag_rgba[4 * o + 3] = 1.0 - fs[b].T;
                }
                if (frag_key) frag_key[o] = (int32_t)fs[b].key;
                if (frag_nsamp) frag_nsamp[o] = fs[b].nsamp;
                if (frag_margin) frag_margin[o] = fs[b].margin;
                ns += fs[b].nsamp;
            }
            if (nsamples) nsamples[k] = ns;
            if (flags) flags[k] = (uint8_t)fl;
        }
        free(fs);
        free(ord);
    }
}

/* Composite arbitrary fragments: per pixel K fragments (premultiplied RGBA
 * and key), non-empty ones in ascending key order, front-to-back over. */
void orc_composite(int npix, int K, const double* frag_rgba, const int32_t* frag_key, double* rgba,
                   uint8_t* order) {
    frag_state* fs = (frag_state*)malloc(sizeof(frag_state) * K);
    uint8_t* ord = (uint8_t*)malloc(K);
    for (int k = 0; k < npix; ++k) {
        for (int b = 0; b < K; ++b) {
            int64_t o = (int64_t)K * k + b;
            for (int a = 0; a < 3; ++a) fs[b].C[a] = frag_rgba[4 * o + a];
            fs[b].T = 1.0 - frag_rgba[4 * o + 3];
            fs[b].key = frag_key[o];
        }
        int m = fragment_order(K, fs, ord);
        orc_rayinfo ri;
        memset(&ri, 0, sizeof ri);
        double out[4], dep;
        composite_pixel(K, fs, &ri, ord, m, out, &dep);
        for (int c = 0; c < 4; ++c) rgba[4 * k + c] = out[c];
        if (order) memcpy(order + (int64_t)K * k, ord, K);
    }
    free(fs);
    free(ord);
}

/* ------------------------------------------------------------------------ */
/* visibility-ordered march with global early termination                    */
/* ------------------------------------------------------------------------ */

/* Reading: the bricks a ray crosses are marched in its front-to-back order,
 * each starting from the transmittance T the bricks in front left, so that
 * C += T alpha c, T *= (1 - alpha) runs over the ray's samples as one march;
 * the march stops after the first sample with 1 - T > ert (global early
 * termination: a brick behind an opaque front is not marched at all).
 * Depth: t of the first sample of the first brick whose segment adds
 * opacity.  With field != NULL the unpartitioned plain definition (the whole
 * float32 field owns every sample); with bricks the owner of each sample
 * evaluates it.  Per listed pixel: rgba, depth, the opacity the depth's
 * segment adds (relative to what reaches it), samples evaluated, flags
 * (EXIT / OWNER / ERT ambiguity as for the sort-last render, the ERT margin
 * taken on the global opacity). */
void orc_render_ordered(const orc_grid* g, const float* field, int K, const orc_brick* bricks, const orc_tf* tf,
                        const orc_camera* cam, const orc_frame* fr, int npix, const int32_t* pix, double* rgba,
                        double* depth, double* depth_alpha, int64_t* nsamples, uint8_t* flags) {
    int all_lo[3] = {0, 0, 0};
    int ert_on = fr->ert > 0.0 && fr->ert < 1.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < npix; ++k) {
        int p = pix ? pix[k] : k;
        orc_rayinfo ri;
        ray_samples(g, cam, fr, p % fr->width, p / fr->width, &ri);
        int fl = ri.flags;
        double C[3] = {0, 0, 0}, T = 1.0, dep = INFINITY, dep_a = 0.0;
        int64_t ns = 0;
        int owner = -1, seg_owner = -1;
        double seg_T0 = 1.0;
        int64_t seg_first = 0;
        for (int64_t j = 0; j < ri.n; ++j) {
            double q[3], tj;
            sample_point(g, &ri, j, q, &tj);
            double s;
            if (bricks) {
                owner = find_owner(g, K, bricks, q, owner);
                if (owner < 0) continue;
                if (near_internal_face(g, &bricks[owner], &ri, tj, fr->amb_samples)) fl |= ORC_FLAG_OWNER_AMBIG;
                int bl[3], bn[3];
                orc_stored_box(g->dims, bricks[owner].owned_lo, bricks[owner].owned_hi, bl, bn);
                s = trilinear(bricks[owner].data, bricks[owner].dtype, bricks[owner].scale, bl, bn, q, NULL, NULL);
            } else {
                owner = 0;
                s = trilinear(field, ORC_F32, 1.0, all_lo, g->dims, q, NULL, NULL);
            }
            if (owner != seg_owner) {          /* a new brick segment begins */
                if (seg_owner >= 0 && isinf(dep) && T < seg_T0) {
                    dep = ri.t_enter + (seg_first + 0.5) * ri.dt;
                    dep_a = 1.0 - T / seg_T0;
                }
                seg_owner = owner;
                seg_T0 = T;
                seg_first = j;
            }
            double c[3], al;
            classify(tf, fr, ri.dt, s, c, &al);
            double A_before = 1.0 - T;
            for (int a = 0; a < 3; ++a) C[a] += T * al * c[a];
            T *= 1.0 - al;
            ++ns;
            if (ert_on && 1.0 - T > fr->ert) {
                double m1 = (1.0 - T) - fr->ert, m0 = fr->ert - A_before;
                if ((m1 < m0 ? m1 : m0) < fr->amb_alpha) fl |= ORC_FLAG_ERT_AMBIG;
                break;
            }
        }
        if (seg_owner >= 0 && isinf(dep) && T < seg_T0) {
            dep = ri.t_enter + (seg_first + 0.5) * ri.dt;
            dep_a = 1.0 - T / seg_T0;
        }
        if (depth_alpha) depth_alpha[k] = dep_a;
        rgba[4 * k + 0] = C[0];
        rgba[4 * k + 1] = C[1];
        rgba[4 * k + 2] = C[2];
        rgba[4 * k + 3] = 1.0 - T;
        if (depth) depth[k] = dep;
        if (nsamples) nsamples[k] = ns;
        if (flags) flags[k] = (uint8_t)fl;
    }
}

/* ------------------------------------------------------------------------ */
/* deep fragments: empty-space skipping splits a brick's segment             */
/* ------------------------------------------------------------------------ */

/* Readings (the paper's compositor accepts several fragments per pixel from
 * one rank, §2.1 and §5.1.1, for parts that are not convex or renderers that
 * emit several segments; it gives no rule for producing them):
 *   - a brick's stored box is cut into macro-cells of ORC_MACRO^3 cells,
 *     macro-cell (mx, my, mz) holding the cells 8 m .. 8 m + 7 per axis (the
 *     last one per axis may hold fewer); its range is the min and max of the
 *     stored values (times the brick's scale) of the nodes its cells touch;
 *   - a macro-cell is transparent when every TF entry a sample inside can
 *     read has opacity exactly 0.  A sample of value v reads entries i0(v)
 *     and i0(v) + 1 (the lookup of tf_lookup); the values inside lie in the
 *     range, so the entries read lie in i0(lo) .. i0(hi) + 1;
 *   - samples in transparent macro-cells have alpha 0 and are not
 *     evaluated.  The brick's segment then splits: each maximal run of
 *     evaluated samples (consecutive in j within the brick) is its own
 *     fragment, premultiplied RGBA over the run, key = j of the run's first
 *     sample.  At most `deep` fragments per brick and pixel: a run after the
 *     last one continues it (compositing it separately would give the same
 *     colour);
 *   - per-fragment early termination stays per brick: the march of a brick
 *     stops after the first sample with 1 - prod(1 - alpha) > ert over all
 *     of the brick's samples so far;
 *   - the composite sorts every fragment of the pixel by key (keys are
 *     distinct) and blends front to back; depth = t of the first sample of
 *     the first fragment with A > 0.
 * Flags, besides the sort-last render's: MACRO_AMBIG where the kernel's
 * FP32 arithmetic could decide a split otherwise -- a sample within
 * 1e-3 node of a face between macro-cells of different transparency, or a
 * sample in a macro-cell whose range ends lie within 2e-6 n of a TF entry
 * boundary (u), where the classification changes if i0 moves by one. */

#define ORC_MACRO 8
#define ORC_DEEP_MAX 16
#define ORC_FLAG_MACRO_AMBIG 32

typedef struct {
    int mn[3];            /* macro-cells per axis */
    uint8_t* empty;       /* 1: transparent */
    uint8_t* amb;         /* 1: classification within the rounding band */
} macro_table;

static double tf_u(const orc_tf* tf, double v) {
    double x = (v - tf->vmin) / (tf->vmax - tf->vmin);
    if (x < 0.0) x = 0.0;
    if (x > 1.0) x = 1.0;
    return x * (tf->n - 1);
}

static int tf_i0(const orc_tf* tf, double u) {
    int i0 = (int)floor(u);
    if (i0 > tf->n - 2) i0 = tf->n - 2;
    if (i0 < 0) i0 = 0;
    return i0;
}

/* entries e0 .. e1 (clamped to the table) all of opacity exactly 0? */
static int tf_zero(const orc_tf* tf, int e0, int e1) {
    if (e0 < 0) e0 = 0;
    if (e1 > tf->n - 1) e1 = tf->n - 1;
    for (int e = e0; e <= e1; ++e)
        if (tf->rgba[4 * e + 3] != 0.0f) return 0;
    return 1;
}

static void macro_build(const orc_grid* g, const orc_brick* b, const orc_tf* tf, macro_table* mt) {
    int bl[3], bn[3];
    orc_stored_box(g->dims, b->owned_lo, b->owned_hi, bl, bn);
    for (int a = 0; a < 3; ++a) mt->mn[a] = (bn[a] - 2) / ORC_MACRO + 1;
    int64_t n = (int64_t)mt->mn[0] * mt->mn[1] * mt->mn[2];
    mt->empty = (uint8_t*)malloc(n);
    mt->amb = (uint8_t*)malloc(n);
    double band = 2e-6 * tf->n;
    for (int mz = 0; mz < mt->mn[2]; ++mz)
        for (int my = 0; my < mt->mn[1]; ++my)
            for (int mx = 0; mx < mt->mn[0]; ++mx) {
                int m0[3] = {mx * ORC_MACRO, my * ORC_MACRO, mz * ORC_MACRO};
                double lo = INFINITY, hi = -INFINITY;
                for (int z = m0[2]; z <= m0[2] + ORC_MACRO && z < bn[2]; ++z)
                    for (int y = m0[1]; y <= m0[1] + ORC_MACRO && y < bn[1]; ++y)
                        for (int x = m0[0]; x <= m0[0] + ORC_MACRO && x < bn[0]; ++x) {
                            double v = b->scale * decode(b->data, b->dtype, ((int64_t)z * bn[1] + y) * bn[0] + x);
                            if (v < lo) lo = v;
                            if (v > hi) hi = v;
                        }
                double ulo = tf_u(tf, lo), uhi = tf_u(tf, hi);
                int e0 = tf_i0(tf, ulo), e1 = tf_i0(tf, uhi) + 1;
                int64_t m = ((int64_t)mz * mt->mn[1] + my) * mt->mn[0] + mx;
                mt->empty[m] = (uint8_t)tf_zero(tf, e0, e1);
                /* an end within the band of an entry boundary: widen by one */
                int w0 = fabs(ulo - nearbyint(ulo)) < band ? e0 - 1 : e0;
                int w1 = fabs(uhi - nearbyint(uhi)) < band ? e1 + 1 : e1;
                mt->amb[m] = (uint8_t)(tf_zero(tf, w0, w1) != mt->empty[m]);
            }
}

static int64_t macro_index(const macro_table* mt, const int c[3]) {
    return ((int64_t)(c[2] / ORC_MACRO) * mt->mn[1] + c[1] / ORC_MACRO) * mt->mn[0] + c[0] / ORC_MACRO;
}

typedef struct {
    double C[ORC_DEEP_MAX][3], T[ORC_DEEP_MAX];
    int64_t key[ORC_DEEP_MAX];
    int nf;               /* fragments started */
    int in_run;           /* the brick's previous sample was evaluated */
    double Tb;            /* transmittance over the brick's samples */
    int done;
    int32_t nsamp;
} deep_state;

/* Deep-fragment render (readings above).  Outputs per listed pixel k (any
 * pointer may be NULL): rgba, depth; frag_rgba[((k K + b) deep + i) 4 ..],
 * frag_key[(k K + b) deep + i] (2^31 - 1 past the brick's count),
 * frag_count[k K + b]; nsamples (evaluated); flags. */
void orc_render_deep(const orc_grid* g, int K, const orc_brick* bricks, const orc_tf* tf, const orc_camera* cam,
                     const orc_frame* fr, int deep, int npix, const int32_t* pix, double* rgba, double* depth,
                     double* frag_rgba, int32_t* frag_key, int32_t* frag_count, int64_t* nsamples,
                     uint8_t* flags) {
    if (deep < 1) deep = 1;
    if (deep > ORC_DEEP_MAX) deep = ORC_DEEP_MAX;
    macro_table* mt = (macro_table*)malloc(sizeof(macro_table) * K);
    for (int b = 0; b < K; ++b) macro_build(g, &bricks[b], tf, &mt[b]);
    int ert_on = fr->ert > 0.0 && fr->ert < 1.0;
#pragma omp parallel
    {
        deep_state* ds = (deep_state*)malloc(sizeof(deep_state) * K);
        int nfr = K * deep;
        int* ob = (int*)malloc(sizeof(int) * nfr);
        int* oi = (int*)malloc(sizeof(int) * nfr);
#pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < npix; ++k) {
            int p = pix ? pix[k] : k;
            orc_rayinfo ri;
            ray_samples(g, cam, fr, p % fr->width, p / fr->width, &ri);
            int fl = ri.flags;
            for (int b = 0; b < K; ++b) {
                ds[b].nf = 0;
                ds[b].in_run = 0;
                ds[b].Tb = 1.0;
                ds[b].done = 0;
                ds[b].nsamp = 0;
            }
            int owner = -1;
            for (int64_t j = 0; j < ri.n; ++j) {
                double q[3], tj;
                sample_point(g, &ri, j, q, &tj);
                owner = find_owner(g, K, bricks, q, owner);
                if (owner < 0) continue;
                const orc_brick* B = &bricks[owner];
                deep_state* f = &ds[owner];
                if (near_internal_face(g, B, &ri, tj, fr->amb_samples)) fl |= ORC_FLAG_OWNER_AMBIG;
                if (f->done) continue;
                int bl[3], bn[3], c[3];
                orc_stored_box(g->dims, B->owned_lo, B->owned_hi, bl, bn);
                for (int a = 0; a < 3; ++a) {
                    int ci = (int)floor(q[a]);
                    if (ci < bl[a]) ci = bl[a];
                    if (ci > bl[a] + bn[a] - 2) ci = bl[a] + bn[a] - 2;
                    c[a] = ci - bl[a];
                }
                const macro_table* M = &mt[owner];
                int64_t m = macro_index(M, c);
                if (M->amb[m]) fl |= ORC_FLAG_MACRO_AMBIG;
                for (int a = 0; a < 3; ++a) {        /* near a face to a macro-cell of the other kind */
                    double ql = q[a] - bl[a];
                    int face = ORC_MACRO * (int)nearbyint(ql / ORC_MACRO);
                    if (face <= 0 || face > bn[a] - 2 || fabs(ql - face) >= 1e-3) continue;
                    int c2[3] = {c[0], c[1], c[2]};
                    c2[a] = c[a] >= face ? face - 1 : face;
                    if (M->empty[macro_index(M, c2)] != M->empty[m]) fl |= ORC_FLAG_MACRO_AMBIG;
                }
                if (M->empty[m]) {
                    f->in_run = 0;
                    continue;
                }
                if (!f->in_run && f->nf < deep) {     /* a new run: a new fragment */
                    int i = f->nf++;
                    f->C[i][0] = f->C[i][1] = f->C[i][2] = 0.0;
                    f->T[i] = 1.0;
                    f->key[i] = j;
                }
                f->in_run = 1;
                int i = f->nf - 1;
                double s = trilinear(B->data, B->dtype, B->scale, bl, bn, q, NULL, NULL);
                double col[3], al;
                classify(tf, fr, ri.dt, s, col, &al);
                double A_before = 1.0 - f->Tb;
                for (int a = 0; a < 3; ++a) f->C[i][a] += f->T[i] * al * col[a];
                f->T[i] *= 1.0 - al;
                f->Tb *= 1.0 - al;
                f->nsamp++;
                if (ert_on && 1.0 - f->Tb > fr->ert) {
                    f->done = 1;
                    double m1 = (1.0 - f->Tb) - fr->ert, m0 = fr->ert - A_before;
                    if ((m1 < m0 ? m1 : m0) < fr->amb_alpha) fl |= ORC_FLAG_ERT_AMBIG;
                }
            }
            /* every fragment of the pixel, by ascending key (insertion sort) */
            int nall = 0;
            for (int b = 0; b < K; ++b)
                for (int i = 0; i < ds[b].nf; ++i) {
                    int at = nall++;
                    while (at > 0 && ds[ob[at - 1]].key[oi[at - 1]] > ds[b].key[i]) {
                        ob[at] = ob[at - 1];
                        oi[at] = oi[at - 1];
                        --at;
                    }
                    ob[at] = b;
                    oi[at] = i;
                }
            double C[3] = {0, 0, 0}, A = 0.0, dep = INFINITY;
            for (int r = 0; r < nall; ++r) {
                const deep_state* f = &ds[ob[r]];
                int i = oi[r];
                double Ak = 1.0 - f->T[i];
                for (int a = 0; a < 3; ++a) C[a] += (1.0 - A) * f->C[i][a];
                A += (1.0 - A) * Ak;
                if (Ak > 0.0 && isinf(dep)) dep = ri.t_enter + (f->key[i] + 0.5) * ri.dt;
            }
            if (rgba) {
                rgba[4 * k + 0] = C[0];
                rgba[4 * k + 1] = C[1];
                rgba[4 * k + 2] = C[2];
                rgba[4 * k + 3] = A;
            }
            if (depth) depth[k] = dep;
            int64_t ns = 0;
            for (int b = 0; b < K; ++b) {
                int64_t o = (int64_t)K * k + b;
                for (int i = 0; i < deep; ++i) {
                    int64_t oo = o * deep + i;
                    int live = i < ds[b].nf;
                    if (frag_rgba)
                        for (int a = 0; a < 4; ++a)
                            frag_rgba[4 * oo + a] = !live ? 0.0 : a < 3 ? ds[b].C[i][a] : 1.0 - ds[b].T[i];
                    if (frag_key) frag_key[oo] = live ? (int32_t)ds[b].key[i] : ORC_KEY_EMPTY;
                }
                if (frag_count) frag_count[o] = ds[b].nf;
                ns += ds[b].nsamp;
            }
            if (nsamples) nsamples[k] = ns;
            if (flags) flags[k] = (uint8_t)fl;
        }
        free(ds);
        free(ob);
        free(oi);
    }
    for (int b = 0; b < K; ++b) {
        free(mt[b].empty);
        free(mt[b].amb);
    }
    free(mt);
}

/* ------------------------------------------------------------------------ */
/* volumetric shadows by ray forwarding                                      */
/* ------------------------------------------------------------------------ */

/* Readings (the global effect compositing cannot produce, §7 and Fig. 6,
 * that data-parallel ray tracers get by forwarding ray wave-fronts between
 * ranks, §2.3; the paper gives no shading equations):
 *   - one directional light, unit direction L toward the light (node and
 *     world directions agree: the spacing is uniform);
 *   - the shadow ray of a sample at node-space point p takes samples at
 *     p + (i + 1/2) h L, i = 0, 1, ..., while they lie in the volume box
 *     [0, dims - 1] (the box is convex and p lies in it, so these are the
 *     first n_s); each attenuates by 1 - alpha_i with
 *     alpha_i = 1 - exp(-sigma_max a(s_i) h spacing), the same emission-
 *     absorption model at step h (node units);
 *   - T_light(p) = prod_i (1 - alpha_i);
 *   - the sample's emitted colour c becomes c (k_a + (1 - k_a) T_light(p)),
 *     k_a the ambient term; opacities and the compositing are unchanged;
 *   - data-parallel form: the primary samples stay with their owner brick
 *     (per-brick fragments, sort-last composite); each shadow sample is
 *     evaluated by the brick owning its position, so T_light is the product
 *     of one partial product per brick the shadow ray crosses (the order
 *     the bricks take does not change it).
 * Flag SHADOW_AMBIG: a shadow sample of an evaluated primary sample lies
 * within 1e-3 node of the box's faces and has alpha > 0 (FP32 positions
 * may count it otherwise). */

#define ORC_FLAG_SHADOW_AMBIG 64

typedef struct {
    double dir[3];        /* unit direction toward the light */
    double step_voxels;   /* h, node units */
    double ambient;       /* k_a */
} orc_light;

/* scalar value at node-space point q: the whole field, or the owner brick */
static double value_at(const orc_grid* g, const float* field, int K, const orc_brick* bricks, const double q[3],
                       int* hint) {
    if (field) {
        int lo[3] = {0, 0, 0};
        return trilinear(field, ORC_F32, 1.0, lo, g->dims, q, NULL, NULL);
    }
    int o = find_owner(g, K, bricks, q, *hint);
    if (o < 0) o = find_owner(g, K, bricks, q, -1);
    *hint = o;
    int bl[3], bn[3];
    orc_stored_box(g->dims, bricks[o].owned_lo, bricks[o].owned_hi, bl, bn);
    return trilinear(bricks[o].data, bricks[o].dtype, bricks[o].scale, bl, bn, q, NULL, NULL);
}

/* signed distance of q to the volume box's faces (negative outside) */
static double box_margin(const orc_grid* g, const double q[3]) {
    double m = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double d0 = q[a], d1 = (g->dims[a] - 1) - q[a];
        if (d0 < m) m = d0;
        if (d1 < m) m = d1;
    }
    return m;
}

static double light_transmittance(const orc_grid* g, const float* field, int K, const orc_brick* bricks,
                                  const orc_tf* tf, const orc_frame* fr, const orc_light* L, const double p[3],
                                  int* amb, int64_t* count) {
    double T = 1.0, hw = L->step_voxels * g->spacing;
    int hint = -1;
    for (int64_t i = 0;; ++i) {
        double q[3];
        for (int a = 0; a < 3; ++a) q[a] = p[a] + (i + 0.5) * L->step_voxels * L->dir[a];
        double m = box_margin(g, q);
        if (fabs(m) < 1e-3) {               /* at a face: does counting it matter? */
            double qc[3], c[3], al;
            for (int a = 0; a < 3; ++a) qc[a] = q[a] < 0.0 ? 0.0 : q[a] > g->dims[a] - 1 ? g->dims[a] - 1 : q[a];
            classify(tf, fr, hw, value_at(g, field, K, bricks, qc, &hint), c, &al);
            if (al > 0.0) *amb = 1;
        }
        if (m < 0.0) break;
        double c[3], al;
        classify(tf, fr, hw, value_at(g, field, K, bricks, q, &hint), c, &al);
        T *= 1.0 - al;
        ++*count;
    }
    return T;
}

/* Shadowed render (readings above).  field != NULL: the plain definition
 * on the whole float32 field (every sample evaluated from it); else the
 * partitioned form: per-brick fragments of the owned primary samples with
 * per-fragment early termination, shadow samples evaluated by their owner
 * bricks, sort-last composite.  Outputs per listed pixel: rgba, depth,
 * primary samples evaluated, shadow samples evaluated (for the primary
 * samples with alpha > 0), flags. */
void orc_render_shadow(const orc_grid* g, const float* field, int K, const orc_brick* bricks, const orc_tf* tf,
                       const orc_camera* cam, const orc_frame* fr, const orc_light* L, int npix,
                       const int32_t* pix, double* rgba, double* depth, int64_t* nsamples, int64_t* nshadow,
                       uint8_t* flags) {
    int ert_on = fr->ert > 0.0 && fr->ert < 1.0 && !field;
    int KK = field ? 1 : K;
#pragma omp parallel
    {
        frag_state* fs = (frag_state*)malloc(sizeof(frag_state) * KK);
        uint8_t* ord = (uint8_t*)malloc(KK);
#pragma omp for schedule(dynamic, 4)
        for (int k = 0; k < npix; ++k) {
            int p = pix ? pix[k] : k;
            orc_rayinfo ri;
            ray_samples(g, cam, fr, p % fr->width, p / fr->width, &ri);
            int fl = ri.flags, amb = 0, owner = -1, hint = -1;
            int64_t nsh = 0;
            for (int b = 0; b < KK; ++b) {
                fs[b].C[0] = fs[b].C[1] = fs[b].C[2] = 0.0;
                fs[b].T = 1.0;
                fs[b].key = ORC_KEY_EMPTY;
                fs[b].nsamp = 0;
                fs[b].done = 0;
            }
            for (int64_t j = 0; j < ri.n; ++j) {
                double q[3], tj;
                sample_point(g, &ri, j, q, &tj);
                if (field) {
                    owner = 0;
                } else {
                    owner = find_owner(g, K, bricks, q, owner);
                    if (owner < 0) continue;
                    if (near_internal_face(g, &bricks[owner], &ri, tj, fr->amb_samples)) fl |= ORC_FLAG_OWNER_AMBIG;
                }
                frag_state* f = &fs[owner];
                if (f->key == ORC_KEY_EMPTY) f->key = j;
                if (f->done) continue;
                hint = owner;
                double s = value_at(g, field, K, bricks, q, &hint);
                double c[3], al;
                classify(tf, fr, ri.dt, s, c, &al);
                if (al > 0.0) {
                    double Tl = light_transmittance(g, field, K, bricks, tf, fr, L, q, &amb, &nsh);
                    double w = L->ambient + (1.0 - L->ambient) * Tl;
                    for (int a = 0; a < 3; ++a) c[a] *= w;
                }
                double A_before = 1.0 - f->T;
                for (int a = 0; a < 3; ++a) f->C[a] += f->T * al * c[a];
                f->T *= 1.0 - al;
                f->nsamp++;
                if (ert_on && 1.0 - f->T > fr->ert) {
                    f->done = 1;
                    double m1 = (1.0 - f->T) - fr->ert, m0 = fr->ert - A_before;
                    if ((m1 < m0 ? m1 : m0) < fr->amb_alpha) fl |= ORC_FLAG_ERT_AMBIG;
                }
            }
            if (amb) fl |= ORC_FLAG_SHADOW_AMBIG;
            int m = fragment_order(KK, fs, ord);
            double out[4], dep;
            composite_pixel(KK, fs, &ri, ord, m, out, &dep);
            for (int c = 0; c < 4; ++c) rgba[4 * k + c] = out[c];
            if (depth) depth[k] = dep;
            int64_t ns = 0;
            for (int b = 0; b < KK; ++b) ns += fs[b].nsamp;
            if (nsamples) nsamples[k] = ns;
            if (nshadow) nshadow[k] = nsh;
            if (flags) flags[k] = (uint8_t)fl;
        }
        free(fs);
        free(ord);
    }
}

/* T_light at arbitrary node-space points (for pins): the field or bricks
 * as above. */
void orc_light_transmittance(const orc_grid* g, const float* field, int K, const orc_brick* bricks,
                             const orc_tf* tf, const orc_frame* fr, const orc_light* L, int n, const double* pts,
                             double* T, int64_t* count, uint8_t* amb) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < n; ++k) {
        int a = 0;
        int64_t c = 0;
        T[k] = light_transmittance(g, field, K, bricks, tf, fr, L, pts + 3 * k, &a, &c);
        if (count) count[k] = c;
        if (amb) amb[k] = (uint8_t)a;
    }
}

/* ------------------------------------------------------------------------ */
/* iso-surface fragments (first hit per brick, depth composite)              */
/* ------------------------------------------------------------------------ */

/* Readings (the paper's z-composited surfaces, its teaser's in-situ
 * iso-surface and the compositing tests of §7; no equations are given):
 *   - the samples are the volume-rendering samples of the ray (t_j, s_j);
 *   - the hit is the first pair (j - 1, j), j >= 1, across which
 *     [s >= iso] changes; h = j;
 *   - the surface point lies at t* = t_{h-1} + f dt with
 *     f = (iso - s_{h-1}) / (s_h - s_{h-1}) (linear between the samples);
 *   - data-parallel form: the brick owning sample j tests the pair
 *     (j - 1, j), evaluating s_{j-1} itself (it lies in its ghost layer),
 *     and keeps its first hit as its fragment; the composite takes the
 *     fragment with the smallest key (opaque surfaces: nearest first);
 *   - colour: TF rgb at iso times 0.25 + 0.75 |N.d| / (|N| |d|), N the
 *     gradient of the trilinear interpolant of the cell holding the surface
 *     point (in the reporting brick), d the ray direction; factor 1 where
 *     N = 0; alpha 1.  No hit: (0, 0, 0, 0) and depth +inf.
 * Flagged ISO_AMBIG (a rounded s or point may decide otherwise): a sample up
 * to the hit (all samples without a hit) within iso_eps of iso, or the
 * surface point within 1e-4 of a cell face; OWNER_AMBIG: a sample up to the
 * hit near an internal brick face. */

/* Gradient of the trilinear interpolant at node-space point q in the cell
 * trilinear() would use (decoded, scaled corners). */
static void trilinear_grad(const void* data, int dtype, double scale, const int b_lo[3], const int b_n[3],
                           const double q[3], double g[3], double frac[3]) {
    int i[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        int c = (int)floor(q[a]);
        if (c < b_lo[a]) c = b_lo[a];
        if (c > b_lo[a] + b_n[a] - 2) c = b_lo[a] + b_n[a] - 2;
        i[a] = c - b_lo[a];
        f[a] = q[a] - c;
        if (frac) frac[a] = f[a];
    }
    double v[8];
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        int64_t k = ((int64_t)(i[2] + dz) * b_n[1] + (i[1] + dy)) * b_n[0] + (i[0] + dx);
        v[c] = scale * decode(data, dtype, k);
    }
    double fx = f[0], fy = f[1], fz = f[2];
    g[0] = (1 - fz) * ((1 - fy) * (v[1] - v[0]) + fy * (v[3] - v[2])) + fz * ((1 - fy) * (v[5] - v[4]) + fy * (v[7] - v[6]));
    g[1] = (1 - fz) * ((1 - fx) * (v[2] - v[0]) + fx * (v[3] - v[1])) + fz * ((1 - fx) * (v[6] - v[4]) + fx * (v[7] - v[5]));
    g[2] = (1 - fy) * ((1 - fx) * (v[4] - v[0]) + fx * (v[5] - v[1])) + fy * ((1 - fx) * (v[6] - v[2]) + fx * (v[7] - v[3]));
}

typedef struct {
    int64_t key;          /* hit sample index h, or -1 */
    double f;             /* fraction between samples h - 1 and h */
    double dsdt;          /* |s_h - s_{h-1}| */
    double rgba[4];
} iso_frag;

/* Value source of a brick (or of the whole field: K = 1, the grid box). */
typedef struct {
    const void* data;
    int dtype;
    double scale;
    int lo[3], n[3];
} iso_src;

static double src_value(const iso_src* b, const double q[3]) {
    return trilinear(b->data, b->dtype, b->scale, b->lo, b->n, q, NULL, NULL);
}

/* Surface colour and cell-face ambiguity of a hit in source b. */
static void iso_shade(const orc_grid* g, const orc_rayinfo* ri, const iso_src* b, const orc_tf* tf, double iso,
                      int64_t h, double f, double rgba[4], int* fl) {
    double t = ri->t_enter + (h - 0.5 + f) * ri->dt;
    double q[3];
    for (int a = 0; a < 3; ++a) {
        q[a] = (ri->o[a] + t * ri->d[a] - g->origin[a]) / g->spacing;
        if (q[a] < 0.0) q[a] = 0.0;
        if (q[a] > g->dims[a] - 1) q[a] = g->dims[a] - 1;
    }
    double gr[3], fr3[3];
    trilinear_grad(b->data, b->dtype, b->scale, b->lo, b->n, q, gr, fr3);
    for (int a = 0; a < 3; ++a)
        if (fr3[a] < 1e-4 || fr3[a] > 1.0 - 1e-4) *fl |= ORC_FLAG_ISO_AMBIG;
    double nn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    double dn = sqrt(ri->d[0] * ri->d[0] + ri->d[1] * ri->d[1] + ri->d[2] * ri->d[2]);
    double k = 1.0;
    if (nn > 0.0) k = 0.25 + 0.75 * fabs(gr[0] * ri->d[0] + gr[1] * ri->d[1] + gr[2] * ri->d[2]) / (nn * dn);
    double v[4];
    tf_lookup(tf, iso, v, NULL, NULL, NULL);
    for (int c = 0; c < 3; ++c) rgba[c] = v[c] * k;
    rgba[3] = 1.0;
}

/* One pixel.  K sources with their owned boxes (bricks), or K = 1 and no
 * bricks (the whole field, which owns every sample).  Outputs the composited
 * colour, depth, key, |s_h - s_{h-1}|, per-brick keys and flags. */
static void iso_pixel(const orc_grid* g, int K, const orc_brick* bricks, const iso_src* src, const orc_tf* tf,
                      const orc_camera* cam, const orc_frame* fr, double iso, double iso_eps, int px, int py,
                      double rgba[4], double* depth, int64_t* key, double* dsdt, int32_t* frag_key, int* flags,
                      iso_frag* fs) {
    orc_rayinfo ri;
    ray_samples(g, cam, fr, px, py, &ri);
    int fl = ri.flags;
    for (int b = 0; b < K; ++b) fs[b].key = -1;
    int owner = -1;
    int64_t first_hit = -1;
    for (int64_t j = 0; j < ri.n; ++j) {
        double q[3], qp[3], tj;
        sample_point(g, &ri, j, q, &tj);
        owner = bricks ? find_owner(g, K, bricks, q, owner) : 0;
        if (owner < 0) continue;
        double s = src_value(&src[owner], q);
        if (first_hit < 0 && fabs(s - iso) < iso_eps) fl |= ORC_FLAG_ISO_AMBIG;
        /* up to the hit, a sample the GPU may give to the neighbour brick
         * (whose per-brick scale differs under fp8 storage) */
        if (first_hit < 0 && bricks && near_internal_face(g, &bricks[owner], &ri, tj, fr->amb_samples))
            fl |= ORC_FLAG_OWNER_AMBIG;
        if (j == 0 || fs[owner].key >= 0) continue;
        sample_point(g, &ri, j - 1, qp, NULL);
        double sp = src_value(&src[owner], qp);       /* s_{j-1} in this brick */
        if ((sp >= iso) != (s >= iso)) {
            iso_frag* fg = &fs[owner];
            fg->key = j;
            fg->f = (iso - sp) / (s - sp);
            fg->dsdt = fabs(s - sp);
            int dummy = 0;
            iso_shade(g, &ri, &src[owner], tf, iso, j, fg->f, fg->rgba, first_hit < 0 ? &fl : &dummy);
            if (first_hit < 0) first_hit = j;
        }
    }
    /* depth composite: the smallest key */
    int best = -1;
    for (int b = 0; b < K; ++b) {
        if (frag_key) frag_key[b] = fs[b].key >= 0 ? (int32_t)fs[b].key : 2147483647;
        if (fs[b].key >= 0 && (best < 0 || fs[b].key < fs[best].key)) best = b;
    }
    if (best >= 0) {
        for (int c = 0; c < 4; ++c) rgba[c] = fs[best].rgba[c];
        *depth = ri.t_enter + (fs[best].key - 0.5 + fs[best].f) * ri.dt;
        *key = fs[best].key;
        *dsdt = fs[best].dsdt;
    } else {
        rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
        *depth = INFINITY;
        *key = -1;
        *dsdt = 0.0;
    }
    *flags = fl;
}

/* Iso-surface render of the whole float32 field (the plain definition) or of
 * the bricks (fragments + depth composite).  Per listed pixel k: rgba[4k..],
 * depth[k], key[k] (-1: no hit), dsdt[k], frag_key[K k + b] (bricks only),
 * flags[k]. */
void orc_render_iso(const orc_grid* g, const float* field, int K, const orc_brick* bricks, const orc_tf* tf,
                    const orc_camera* cam, const orc_frame* fr, double iso, double iso_eps, int npix,
                    const int32_t* pix, double* rgba, double* depth, int64_t* key, double* dsdt, int32_t* frag_key,
                    uint8_t* flags) {
    int nsrc = bricks ? K : 1;
    iso_src* src = (iso_src*)malloc(sizeof(iso_src) * nsrc);
    for (int b = 0; b < nsrc; ++b) {
        if (bricks) {
            src[b].data = bricks[b].data;
            src[b].dtype = bricks[b].dtype;
            src[b].scale = bricks[b].scale;
            orc_stored_box(g->dims, bricks[b].owned_lo, bricks[b].owned_hi, src[b].lo, src[b].n);
        } else {
            src[b].data = field;
            src[b].dtype = ORC_F32;
            src[b].scale = 1.0;
            for (int a = 0; a < 3; ++a) {
                src[b].lo[a] = 0;
                src[b].n[a] = g->dims[a];
            }
        }
    }
#pragma omp parallel
    {
        iso_frag* fs = (iso_frag*)malloc(sizeof(iso_frag) * nsrc);
#pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < npix; ++k) {
            int p = pix ? pix[k] : k;
            int fl = 0;
            int64_t kk;
            double ds, dep;
            iso_pixel(g, nsrc, bricks, src, tf, cam, fr, iso, iso_eps, p % fr->width, p / fr->width,
                      rgba + 4 * (int64_t)k, &dep, &kk, &ds, frag_key && bricks ? frag_key + (int64_t)K * k : NULL,
                      &fl, fs);
            if (depth) depth[k] = dep;
            if (key) key[k] = kk;
            if (dsdt) dsdt[k] = ds;
            if (flags) flags[k] = (uint8_t)fl;
        }
        free(fs);
    }
    free(src);
}

/* ------------------------------------------------------------------------ */
/* k-d visibility order                                                      */
/* ------------------------------------------------------------------------ */

/* Front-to-back order of the leaves of a k-d tree seen from a point: at each
 * node visit first the child on the eye's side of the split plane (node-space
 * coordinate split - 1/2), the lower child when the eye lies on the plane.
 * A child < 0 is leaf -(rank + 1).  Empty tree: the single rank 0. */
static int kd_visit(int node, const int* axis, const int* split, const int* left, const int* right,
                    const double eye_q[3], uint8_t* out, int m) {
    if (node < 0) {
        out[m] = (uint8_t)(-node - 1);
        return m + 1;
    }
    double plane = split[node] - 0.5;
    int first = eye_q[axis[node]] > plane ? right[node] : left[node];
    int second = first == right[node] ? left[node] : right[node];
    m = kd_visit(first, axis, split, left, right, eye_q, out, m);
    return kd_visit(second, axis, split, left, right, eye_q, out, m);
}

int orc_kd_order(int nnodes, const int* axis, const int* split, const int* left, const int* right,
                 const double eye_q[3], uint8_t* out) {
    if (nnodes == 0) {
        out[0] = 0;
        return 1;
    }
    return kd_visit(0, axis, split, left, right, eye_q, out, 0);
}

/* ------------------------------------------------------------------------ */
/* gradients: reverse mode with a per-sample tape                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int brick;
    double s, alpha, c[3];
    int i0;
    double w, duds, u;   /* u: (s - vmin) / (vmax - vmin) (N - 1), not clamped */
    int flat;            /* all 8 corner values equal: s is exact in any arithmetic */
    double vlo, vhi;     /* smallest and largest corner value */
    int64_t idx[8];
    double wt[8];
} tape_entry;

/* Slope d(Tab[k+1][c] - Tab[k][c]) du/ds of channel c on TF segment k, with
 * the segments outside [0, N - 2] standing for the clamped ends (slope 0). */
static double seg_slope(const orc_tf* tf, int k, int c) {
    if (k < 0 || k > tf->n - 2) return 0.0;
    return (tf->rgba[4 * (k + 1) + c] - tf->rgba[4 * k + c]) * (double)(tf->n - 1) / (tf->vmax - tf->vmin);
}

/* Reverse-mode gradient of sum_k <g_k, I_k> over listed pixels, where I_k is
 * the partitioned render (fragments + composite, ERT as in the forward).
 * Differentiates with respect to the TF table (dtf: n x 4, accumulated) and
 * the global field values (dvol: global nodes, accumulated; a ghost copy's
 * gradient goes to its global node).  The field enters through each brick's
 * stored values times its scale.  Reverse sweep of the recurrences, no
 * closed-form adjoint:
 *   over:  C' = C + (1 - A) C_k,  A' = A + (1 - A) A_k
 *   EA:    C' = C + T alpha c,    T' = T (1 - alpha),  A_k = 1 - T_end
 *   alpha = 1 - exp(-sigma_max a dt);  TF lerp;  trilinear.
 *
 * Knot ambiguity (optional damb, global nodes, accumulated): the lerp is not
 * differentiable in s at a knot where the slope changes; there the gradient
 * takes the segment to the right (the left one at u = N - 1).  A sample
 * whose u = (s - vmin) / (vmax - vmin) (N - 1) lies within knot_eps of a
 * knot m is one a rounded s may place on either side of m, and either
 * one-sided derivative is then a correct answer.  A sample whose eight
 * corner values are equal is the exception: any interpolation by convex
 * combinations returns that value exactly, so it cannot change sides.  At
 * the two end knots the other side is the clamp (slope 0), which a sample
 * reaches only if s can leave [vmin, vmax]; interpolation by convex
 * combinations keeps s within its corners' range, so only samples with a
 * corner outside [vmin, vmax] count there.  For the other samples near a
 * knot damb
 * collects, per voxel, |ds-adjoint with the other segment - with the chosen
 * one| times the trilinear weight: how far a correct gradient may lie from
 * dvol.  Both sides of m use the same value adjoints, since the TF value is
 * continuous there.
 *
 * TF-coordinate ambiguity (optional dtf_amb, n x 4, accumulated): a sample
 * splits its value adjoint g between entries i0 and i0 + 1 with weights
 * 1 - w and w, w = u - i0.  An FP32 u carries about 3 roundings of 2^-24 u
 * (the sample value, the scale, the product), so w may move by
 * du = 2^-22 max(u, 1), which moves each of the two entries by du |g|
 * (per channel); past a knot the same du moves the sample's weight between
 * neighbouring entries by the same amount.  dtf_amb sums du |g| over the
 * samples: how far a correct TF gradient may lie from dtf. */
void orc_grad_bricks(const orc_grid* g, int K, const orc_brick* bricks, const orc_tf* tf, const orc_camera* cam,
                     const orc_frame* fr, int npix, const int32_t* pix, const double* grad_rgba, double* dtf,
                     double* dvol, double* damb, double knot_eps, double* dtf_amb) {
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double* dtf_priv = (double*)calloc((size_t)nthreads * tf->n * 4, sizeof(double));
    double* amb_priv = dtf_amb ? (double*)calloc((size_t)nthreads * tf->n * 4, sizeof(double)) : NULL;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* my_dtf = dtf_priv + (size_t)tid * tf->n * 4;
        double* my_amb = amb_priv ? amb_priv + (size_t)tid * tf->n * 4 : NULL;
        frag_state* fs = (frag_state*)malloc(sizeof(frag_state) * K);
        uint8_t* ord = (uint8_t*)malloc(K);
        size_t cap = 1024;
        tape_entry* tape = (tape_entry*)malloc(cap * sizeof(tape_entry));
        int64_t* perm = (int64_t*)malloc(cap * sizeof(int64_t));
        int64_t* first = (int64_t*)malloc(sizeof(int64_t) * K);
        int64_t* count = (int64_t*)malloc(sizeof(int64_t) * K);
        int* bl = (int*)malloc(sizeof(int) * 3 * K);
        int* bn = (int*)malloc(sizeof(int) * 3 * K);
        for (int b = 0; b < K; ++b) orc_stored_box(g->dims, bricks[b].owned_lo, bricks[b].owned_hi, bl + 3 * b, bn + 3 * b);
#pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < npix; ++k) {
            int p = pix ? pix[k] : k;
            orc_rayinfo ri;
            ray_samples(g, cam, fr, p % fr->width, p / fr->width, &ri);
            /* forward with a tape: record evaluated samples grouped per brick */
            if ((size_t)ri.n > cap) {
                cap = (size_t)ri.n;
                tape = (tape_entry*)realloc(tape, cap * sizeof(tape_entry));
                perm = (int64_t*)realloc(perm, cap * sizeof(int64_t));
            }
            int fl = 0;
            pixel_fragments(g, K, bricks, tf, fr, &ri, fs, &fl);
            /* re-walk the ray and tape the samples each brick evaluated, in ray order */
            int64_t nt = 0;
            for (int b = 0; b < K; ++b) count[b] = 0;
            int owner = -1;
            for (int64_t j = 0; j < ri.n; ++j) {
                double q[3];
                sample_point(g, &ri, j, q, NULL);
                owner = find_owner(g, K, bricks, q, owner);
                if (owner < 0) continue;
                if (count[owner] >= fs[owner].nsamp) continue;   /* after early termination */
                tape_entry* e = &tape[nt++];
                e->brick = owner;
                e->s = trilinear(bricks[owner].data, bricks[owner].dtype, bricks[owner].scale, bl + 3 * owner,
                                 bn + 3 * owner, q, e->idx, e->wt);
                double v[4];
                tf_lookup(tf, e->s, v, &e->i0, &e->w, &e->duds);
                e->u = (e->s - tf->vmin) / (tf->vmax - tf->vmin) * (double)(tf->n - 1);
                e->vlo = e->vhi = bricks[owner].scale * decode(bricks[owner].data, bricks[owner].dtype, e->idx[0]);
                for (int c = 1; c < 8; ++c) {
                    double vc = bricks[owner].scale * decode(bricks[owner].data, bricks[owner].dtype, e->idx[c]);
                    if (vc < e->vlo) e->vlo = vc;
                    if (vc > e->vhi) e->vhi = vc;
                }
                e->flat = e->vlo == e->vhi;
                e->c[0] = v[0]; e->c[1] = v[1]; e->c[2] = v[2];
                e->alpha = 1.0 - exp(-fr->sigma_max * v[3] * ri.dt);
                count[owner]++;
            }
            /* group the tape by brick, keeping ray order within a brick */
            int64_t acc = 0;
            for (int b = 0; b < K; ++b) { first[b] = acc; acc += count[b]; count[b] = 0; }
            for (int64_t i = 0; i < nt; ++i) {
                int b = tape[i].brick;
                perm[first[b] + count[b]++] = i;
            }
            int m = fragment_order(K, fs, ord);
            /* composite forward states A before each fragment */
            double gr[4];
            for (int c = 0; c < 4; ++c) gr[c] = grad_rgba[4 * k + c];
            double Aprev[256];
            double A = 0.0;
            for (int i = 0; i < m; ++i) {
                Aprev[i] = A;
                A += (1.0 - A) * (1.0 - fs[ord[i]].T);
            }
            /* reverse through the over operator */
            double gC[3] = {gr[0], gr[1], gr[2]}, gA = gr[3];
            for (int i = m - 1; i >= 0; --i) {
                const frag_state* f = &fs[ord[i]];
                double Ak = 1.0 - f->T, Ain = Aprev[i];
                double gCk[3], gAk;
                for (int a = 0; a < 3; ++a) gCk[a] = (1.0 - Ain) * gC[a];
                gAk = (1.0 - Ain) * gA;
                double gAin = gA * (1.0 - Ak) - (gC[0] * f->C[0] + gC[1] * f->C[1] + gC[2] * f->C[2]);
                gA = gAin;
                /* reverse through the fragment's EA recurrence */
                int b = ord[i];
                int64_t n0 = first[b], nb = count[b];
                if (nb == 0) continue;
                /* forward transmittances */
                double* Ts = (double*)malloc(sizeof(double) * (nb + 1));
                Ts[0] = 1.0;
                for (int64_t s = 0; s < nb; ++s) Ts[s + 1] = Ts[s] * (1.0 - tape[perm[n0 + s]].alpha);
                double gT = -gAk;   /* A_k = 1 - T_end */
                for (int64_t s = nb - 1; s >= 0; --s) {
                    tape_entry* e = &tape[perm[n0 + s]];
                    double T = Ts[s];
                    double galpha = (gCk[0] * e->c[0] + gCk[1] * e->c[1] + gCk[2] * e->c[2]) * T - gT * T;
                    double gc[3];
                    for (int a = 0; a < 3; ++a) gc[a] = gCk[a] * T * e->alpha;
                    gT = (gCk[0] * e->c[0] + gCk[1] * e->c[1] + gCk[2] * e->c[2]) * e->alpha + gT * (1.0 - e->alpha);
                    /* alpha = 1 - exp(-sigma_max a dt) */
                    double ga = galpha * fr->sigma_max * ri.dt * (1.0 - e->alpha);
                    double gv[4] = {gc[0], gc[1], gc[2], ga};
                    double gw = 0.0;
                    for (int c = 0; c < 4; ++c) {
                        my_dtf[4 * e->i0 + c] += (1.0 - e->w) * gv[c];
                        my_dtf[4 * (e->i0 + 1) + c] += e->w * gv[c];
                        gw += gv[c] * (tf->rgba[4 * (e->i0 + 1) + c] - tf->rgba[4 * e->i0 + c]);
                    }
                    if (my_amb) {
                        double du = ldexp(e->u > 1.0 ? e->u : 1.0, -22);
                        for (int c = 0; c < 4; ++c) {
                            my_amb[4 * e->i0 + c] += du * fabs(gv[c]);
                            my_amb[4 * (e->i0 + 1) + c] += du * fabs(gv[c]);
                        }
                    }
                    double gs = gw * e->duds;
                    double gs_amb = 0.0;
                    if (damb) {
                        double m = floor(e->u + 0.5);
                        if (!e->flat && fabs(e->u - m) < knot_eps) {
                            /* segment the gradient took, and the other one at knot m */
                            int chosen = e->duds == 0.0 ? (e->u < 0.0 ? -1 : tf->n - 1) : e->i0;
                            int other = chosen == (int)m ? (int)m - 1 : (int)m;
                            /* the clamped side of an end knot is out of reach
                             * while every corner lies inside [vmin, vmax] */
                            int reach = 1;
                            if (other < 0 && e->vlo >= tf->vmin) reach = 0;
                            if (other > tf->n - 2 && e->vhi <= tf->vmax) reach = 0;
                            double galt = 0.0;
                            for (int c = 0; c < 4; ++c) galt += gv[c] * seg_slope(tf, other, c);
                            if (reach) gs_amb = fabs(galt - gs);
                        }
                    }
                    if (damb && gs_amb != 0.0) {
                        const int* lo = bl + 3 * e->brick;
                        const int* nn = bn + 3 * e->brick;
                        for (int c = 0; c < 8; ++c) {
                            int64_t li = e->idx[c];
                            int x = (int)(li % nn[0]), y = (int)((li / nn[0]) % nn[1]), z = (int)(li / ((int64_t)nn[0] * nn[1]));
                            int64_t gi = ((int64_t)(z + lo[2]) * g->dims[1] + (y + lo[1])) * g->dims[0] + (x + lo[0]);
                            double contrib = gs_amb * e->wt[c] * fabs((double)bricks[e->brick].scale);
#pragma omp atomic
                            damb[gi] += contrib;
                        }
                    }
                    if (dvol && gs != 0.0) {
                        const int* lo = bl + 3 * e->brick;
                        const int* nn = bn + 3 * e->brick;
                        for (int c = 0; c < 8; ++c) {
                            int64_t li = e->idx[c];
                            int x = (int)(li % nn[0]), y = (int)((li / nn[0]) % nn[1]), z = (int)(li / ((int64_t)nn[0] * nn[1]));
                            int64_t gi = ((int64_t)(z + lo[2]) * g->dims[1] + (y + lo[1])) * g->dims[0] + (x + lo[0]);
                            double contrib = gs * e->wt[c] * bricks[e->brick].scale;
#pragma omp atomic
                            dvol[gi] += contrib;
                        }
                    }
                }
                free(Ts);
            }
        }
        free(fs); free(ord); free(tape); free(perm); free(first); free(count); free(bl); free(bn);
    }
    for (int t = 0; t < nthreads; ++t)
        for (int i = 0; i < tf->n * 4; ++i) {
            dtf[i] += dtf_priv[(size_t)t * tf->n * 4 + i];
            if (dtf_amb) dtf_amb[i] += amb_priv[(size_t)t * tf->n * 4 + i];
        }
    free(dtf_priv);
    free(amb_priv);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
