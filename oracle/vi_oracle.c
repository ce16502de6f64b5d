/*
 * vi_oracle.c -- FP64 CPU oracle of slice-based illuminated ray casting
 * (D. Luo, "Interactive volume illumination of slice-based ray casting",
 * arXiv 2008.06134).
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA library.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it; the library never calls it and there is no CPU fallback built on it.  It
 * shares no code, header or table with the CUDA path.
 *
 * It is plain and slow on purpose: every step follows the paper's order and
 * notation with no blocking, fusion or reordering beyond a parallel loop over
 * independent texels / pixels.
 *
 *   Section 3.2.1, Algorithm 1 -- attenuation buffer built slice by slice,
 *                    nearest slice to the light first (orc_build_stack).
 *   Eq. 8        -- min/max of L.V over the unit cube's vertices.
 *   Eq. 9        -- slice index of a sample, n (L.S - min) / (max - min).
 *   Eq. 10       -- shadow-map (light-space) coordinates of a sample.
 *   Section 3.2.3 -- shell (6 neighbours) and cone (8 points, Eq. 11
 *                    rotation of B_proj about L) scattering coefficients.
 *   Eq. 2, Eq. 3 -- emission-absorption compositing, front to back.
 *   Eq. 7        -- per-sample attenuation coefficient weighting emission.
 *   Eq. 1        -- exact transmittance exp(-integral of kappa) along the
 *                   light ray (orc_transmittance_bruteforce, convergence pin).
 *
 * Variants (all off by default):
 *   Eq. 5-6      -- extinction form: the buffer holds the optical depth
 *                   D_k = sum_{j<k} tau_j, tau_j = -ln(1 - alpha_j), capped at
 *                   ORC_DEPTH_MAX; a lookup's light factor is exp(-D).
 *   slice_filter -- linear interpolation in lambda between the two slices
 *                   bracketing a sample instead of the nearest slice.
 *   shell_count  -- several shells (Section 3.2.3: the number and size of
 *                   the shells can vary) at radii r, 2r, ..., equal weights.
 *   point light  -- a light at a position P (the paper speaks of a light
 *                   position, Fig. 7): light travels along rays from P; the
 *                   slices are planes perpendicular to the axis from P to the
 *                   cube centre, and each texel column is one ray from P
 *                   through a perspective texel grid (orc_point_light_setup).
 *
 * Precision.  Everything whose rounding decides an integer -- the light and
 * camera set-up, sample positions t_i and the count of samples on a ray, the
 * slice index k, the texel cell, the voxel cell and the inside-the-cube test of
 * the sweep -- is computed in IEEE binary32 with the fixed operation order
 * written below (the "index path"; fmaf is a single rounding).  The library
 * computes the same binary32 values independently, so those integers agree bit
 * for bit.  All other arithmetic (interpolation weights, transfer function,
 * attenuation products, scattering averages, compositing) is binary64.
 *
 * Build: cc -std=c11 -O2 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
 * (-ffp-contract=off matters: a contracted a*b+c would change index-path bits.)
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_U8 = 0, ORC_U16 = 1 };
enum { ORC_NONE = 0, ORC_SHADOW = 1, ORC_SHELL = 2, ORC_CONE = 3 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };
enum { ORC_TRANSMITTANCE = 0, ORC_OPTICAL_DEPTH = 1 };
enum { ORC_SLICE_NEAREST = 0, ORC_SLICE_LINEAR = 1 };

/* Cap of the stored optical depth: exp(-64) < 2e-28, zero for every purpose,
   and the cap keeps an opaque texel (tau = infinity) finite for
   interpolation. */
#define ORC_DEPTH_MAX 64.0
#define ORC_MAX_SHELLS 4
#define ORC_MAX_NB (6 * ORC_MAX_SHELLS)

#define ORC_TRACE_WORDS 40
#define ORC_TRACE_NONE 0x7fffffff

typedef struct {
    const void* data; /* vol[z][y][x], x fastest */
    int dtype;        /* ORC_U8 or ORC_U16 */
    int nx, ny, nz;
} orc_volume;

typedef struct {
    const float* rgba; /* M entries of straight RGBA */
    int M;
    float vmin, vmax;
} orc_tf;

/* Light set-up (index path, binary32). */
typedef struct {
    float L[3];     /* unit direction the light travels */
    float min, max; /* Eq. 8 */
    float dL;       /* slice spacing (max - min) / n */
    float kappa;    /* n / (max - min), the ratio of Eq. 9 */
    float Lc;       /* L . c, c the cube centre */
    float U[3], V[3]; /* light-plane basis, V = L x U */
    float h;        /* half extent of the light square about c */
    float sigma;    /* texels per world unit, R / (2 h) */
    float rho0;     /* (R - 1) / 2 */
    int n, R;
    int axis;       /* world axis U was built from */
    int point;      /* 0: directional light L; 1: point light at P, L its axis */
    float P[3];     /* point light position */
} orc_light;

typedef struct {
    int opacity_correction; /* alpha' = 1 - (1 - alpha)^(slice spacing in voxels) */
    float comp_n;           /* darkening compensation exponent, 0 = off */
    int quantity;           /* ORC_TRANSMITTANCE or ORC_OPTICAL_DEPTH */
} orc_build_opts;

typedef struct {
    float eye[3], target[3], up[3];
    int perspective;
    float fovy_deg;
    float ortho_half_height;
} orc_camera;

typedef struct {
    int mode;                   /* ORC_NONE .. ORC_CONE */
    float ert;                  /* stop once A > ert; 2 disables */
    float bg[4];
    float color[3];             /* light colour */
    float ambient;              /* light factor = ambient + (1 - ambient) a_s */
    float step_vox;             /* sample step in voxels */
    int opacity_correction;     /* alpha' = 1 - (1 - alpha)^step_vox */
    float cone_half_angle_deg;  /* cone half angle phi */
    float shell_radius_vox;     /* shell radius r in voxels */
    double ert_band;            /* |A - ert| <= band marks an ERT-ambiguous pixel */
    int quantity;               /* what the buffer holds: ORC_TRANSMITTANCE / ORC_OPTICAL_DEPTH */
    int slice_filter;           /* ORC_SLICE_NEAREST or ORC_SLICE_LINEAR */
    int shell_count;            /* shells at r, 2r, ...; 0 means 1 */
} orc_render_opts;

/* Camera frame (index path, binary32). */
typedef struct {
    float eye[3], f[3], r[3], u[3];
    float sx, sy;
    float dt;
    int perspective, W, H, Nmax;
} orc_frame;

/* One eye ray (index path, binary32). */
typedef struct {
    int hit;
    float o[3], d[3];
    float t0, t1;
    float lo[3], ld[3]; /* (lambda, tu, tv) at t = 0 and their rate per unit t */
    int nnb;
    float nb[ORC_MAX_NB][3]; /* neighbour offsets in (lambda, tu, tv) */
} orc_ray;

/* ------------------------------------------------------------------ */
/* Threads: a plain parallel loop over independent items.             */

static int g_threads = 0;

int orc_set_threads(int n) {
    g_threads = n;
    return 0;
}

int orc_get_threads(void) {
    if (g_threads > 0) return g_threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

typedef void (*orc_task)(void* ctx, long lo, long hi);

typedef struct {
    long n, next, chunk;
    orc_task fn;
    void* ctx;
    pthread_mutex_t mu;
} pf_state;

static void* pf_worker(void* p) {
    pf_state* s = (pf_state*)p;
    for (;;) {
        pthread_mutex_lock(&s->mu);
        long lo = s->next;
        s->next += s->chunk;
        pthread_mutex_unlock(&s->mu);
        if (lo >= s->n) break;
        long hi = lo + s->chunk < s->n ? lo + s->chunk : s->n;
        s->fn(s->ctx, lo, hi);
    }
    return NULL;
}

static void parallel_for(long n, long chunk, orc_task fn, void* ctx) {
    int nt = orc_get_threads();
    if (nt <= 1 || n <= chunk) {
        fn(ctx, 0, n);
        return;
    }
    if (nt > 256) nt = 256;
    pf_state s;
    s.n = n;
    s.next = 0;
    s.chunk = chunk;
    s.fn = fn;
    s.ctx = ctx;
    pthread_mutex_init(&s.mu, NULL);
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < nt - 1; ++t)
        if (pthread_create(&th[started], NULL, pf_worker, &s) == 0) ++started;
    pf_worker(&s);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&s.mu);
}

/* ------------------------------------------------------------------ */
/* Index-path helpers (binary32, one rounding per written operation).  */

static float dot3f(const float a[3], const float b[3]) {
    float p0 = a[0] * b[0];
    float p1 = a[1] * b[1];
    float p2 = a[2] * b[2];
    float s = p0 + p1;
    return s + p2;
}

static void cross3f(const float a[3], const float b[3], float out[3]) {
    float p, q;
    p = a[1] * b[2]; q = a[2] * b[1]; out[0] = p - q;
    p = a[2] * b[0]; q = a[0] * b[2]; out[1] = p - q;
    p = a[0] * b[1]; q = a[1] * b[0]; out[2] = p - q;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor(x) clamped to [lo, hi] and converted to int. */
static int floor_clamp(float x, int lo, int hi) {
    float f = floorf(x);
    if (f < (float)lo) return lo;
    if (f > (float)hi) return hi;
    return (int)f;
}

/* ------------------------------------------------------------------ */
/* Light set-up: Eq. 8 and the light-space frame of Eq. 10.           */

int orc_light_setup(const float dir[3], int n, int R, orc_light* o) {
    if (!dir || !o || n < 1 || R < 1) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(dir[a])) return ORC_EINVAL;
    float len = sqrtf(dot3f(dir, dir));
    if (!(len > 0.0f) || !isfinite(len)) return ORC_EINVAL;
    memset(o, 0, sizeof(*o));
    for (int a = 0; a < 3; ++a) o->L[a] = dir[a] / len;

    /* Eq. 8: min and max of L . V[i] over the eight vertices of [0,1]^3. */
    float mn = 0.0f, mx = 0.0f;
    for (int c = 0; c < 8; ++c) {
        float V[3] = {(float)(c & 1), (float)((c >> 1) & 1), (float)((c >> 2) & 1)};
        float d = dot3f(o->L, V);
        if (c == 0 || d < mn) mn = d;
        if (c == 0 || d > mx) mx = d;
    }
    o->min = mn;
    o->max = mx;
    /* Slice k lies at min + k (max - min) / n (Section 3.2.1); Eq. 9's ratio. */
    float span = mx - mn;
    o->dL = span / (float)n;
    o->kappa = (float)n / span;
    const float c3[3] = {0.5f, 0.5f, 0.5f};
    o->Lc = dot3f(o->L, c3);

    /* Light-space frame (the view matrix L_v of Eq. 10): U from the world axis
       least aligned with L (lowest index on ties), V = L x U. */
    int ax = 0;
    if (fabsf(o->L[1]) < fabsf(o->L[ax])) ax = 1;
    if (fabsf(o->L[2]) < fabsf(o->L[ax])) ax = 2;
    o->axis = ax;
    float w[3];
    for (int b = 0; b < 3; ++b) {
        float e = (b == ax) ? 1.0f : 0.0f;
        float p = o->L[ax] * o->L[b];
        w[b] = e - p;
    }
    float wn = sqrtf(dot3f(w, w));
    for (int b = 0; b < 3; ++b) o->U[b] = w[b] / wn;
    cross3f(o->L, o->U, o->V);

    /* Orthographic light projection L_p: a square of half extent sqrt(3)/2
       about the centre, which holds the cube's shadow for every L. */
    o->h = 0x1.bb67aep-1f;
    float two_h = 2.0f * o->h;
    o->sigma = (float)R / two_h;
    o->rho0 = 0.5f * (float)(R - 1);
    o->n = n;
    o->R = R;
    return ORC_OK;
}

/* Point light at P (f4): L is the axis from P to the centre c, the slices are
   planes perpendicular to L at depths min + k (max - min) / n from P, where
   min / max are the extreme depths (V - P).L of the cube's vertices, and the
   texel grid is perspective: texel (i, j) is the ray from P through
   L + u U + v V with u, v in [-g, g], g the tangent of the half angle of the
   cone from P that holds the cube's circumscribed sphere.  P must be at least
   1 from c (outside that sphere).  U, V as for a directional light along L. */
int orc_point_light_setup(const float pos[3], int n, int R, orc_light* o) {
    if (!pos || !o || n < 1 || R < 1) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(pos[a])) return ORC_EINVAL;
    float q[3] = {0.5f - pos[0], 0.5f - pos[1], 0.5f - pos[2]};
    float dc2 = dot3f(q, q);
    float dc = sqrtf(dc2);
    if (!(dc >= 1.0f) || !isfinite(dc)) return ORC_EINVAL;
    /* The frame of a directional light along the axis; then the depths. */
    int rc = orc_light_setup(q, n, R, o);
    if (rc) return rc;
    o->point = 1;
    for (int a = 0; a < 3; ++a) o->P[a] = pos[a];
    float pa = dot3f(o->L, pos);
    float mn = 0.0f, mx = 0.0f;
    for (int c = 0; c < 8; ++c) {
        float V[3] = {(float)(c & 1), (float)((c >> 1) & 1), (float)((c >> 2) & 1)};
        float d = dot3f(o->L, V) - pa;
        if (c == 0 || d < mn) mn = d;
        if (c == 0 || d > mx) mx = d;
    }
    o->min = mn;
    o->max = mx;
    float span = mx - mn;
    o->dL = span / (float)n;
    o->kappa = (float)n / span;
    o->Lc = 0.0f;
    /* Half extent of the texel grid at unit depth: tan of the half angle of
       the cone tangent to the sphere of radius sqrt(3)/2 about c. */
    float hs = 0x1.bb67aep-1f;
    float hs2 = hs * hs;
    o->h = hs / sqrtf(dc2 - hs2);
    float two_h = 2.0f * o->h;
    o->sigma = (float)R / two_h;
    return ORC_OK;
}

/* World position of texel (i, j) of slice plane k (index path). */
static void texel_world(const orc_light* lt, int i, int j, float sk, float P[3]) {
    float qi = (float)(2 * i + 1) / (float)lt->R;
    float qj = (float)(2 * j + 1) / (float)lt->R;
    float u = (qi - 1.0f) * lt->h;
    float v = (qj - 1.0f) * lt->h;
    if (lt->point) {
        /* The column is the ray from the light through (u, v) on the plane at
           unit depth: w = L + u U + v V; plane k lies at depth sk along L. */
        for (int a = 0; a < 3; ++a) {
            float w0 = fmaf(u, lt->U[a], lt->L[a]);
            float w = fmaf(v, lt->V[a], w0);
            P[a] = fmaf(sk, w, lt->P[a]);
        }
        return;
    }
    for (int a = 0; a < 3; ++a) {
        float b0 = fmaf(u, lt->U[a], 0.5f);
        float b1 = fmaf(v, lt->V[a], b0);
        P[a] = fmaf(sk, lt->L[a], b1);
    }
}

/* Length of a point light's texel column direction w (for opacity
   correction along the column). */
static double column_stretch(const orc_light* lt, int i, int j) {
    if (!lt->point) return 1.0;
    float qi = (float)(2 * i + 1) / (float)lt->R;
    float qj = (float)(2 * j + 1) / (float)lt->R;
    float u = (qi - 1.0f) * lt->h;
    float v = (qj - 1.0f) * lt->h;
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double w = (double)fmaf(v, lt->V[a], fmaf(u, lt->U[a], lt->L[a]));
        s += w * w;
    }
    return sqrt(s);
}

/* Signed distance of slice plane k from the centre along L (index path). */
static float slice_offset(const orc_light* lt, int k) {
    float dk = fmaf((float)k, lt->dL, lt->min);
    return dk - lt->Lc;
}

/* ------------------------------------------------------------------ */
/* Volume reconstruction and classification (binary64).                */

static double voxel(const orc_volume* v, int x, int y, int z) {
    size_t idx = ((size_t)z * (size_t)v->ny + (size_t)y) * (size_t)v->nx + (size_t)x;
    if (v->dtype == ORC_U8) return (double)((const uint8_t*)v->data)[idx];
    return (double)((const uint16_t*)v->data)[idx];
}

/* Trilinear reconstruction at P in [0,1]^3; voxel centres at (idx + 1/2) / N,
   clamp to edge.  The cell (index path) is returned through cell[]. */
static double sample_volume(const orc_volume* v, const float P[3], int cell[3]) {
    const int N[3] = {v->nx, v->ny, v->nz};
    int lo[3], hi[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        float x = fmaf(P[a], (float)N[a], -0.5f);
        int c = floor_clamp(x, -1, N[a]);
        cell[a] = c;
        f[a] = (double)x - floor((double)x);
        lo[a] = clampi(c, 0, N[a] - 1);
        hi[a] = clampi(c + 1, 0, N[a] - 1);
    }
    double acc = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
        int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        double w = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);
        acc += w * voxel(v, bx ? hi[0] : lo[0], by ? hi[1] : lo[1], bz ? hi[2] : lo[2]);
    }
    return acc;
}

/* Same reconstruction at a binary64 position (used by the exact light march). */
static double sample_volume_f64(const orc_volume* v, const double P[3]) {
    const int N[3] = {v->nx, v->ny, v->nz};
    int lo[3], hi[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double x = P[a] * (double)N[a] - 0.5;
        double fl = floor(x);
        f[a] = x - fl;
        int c = fl < -1.0 ? -1 : (fl > (double)N[a] ? N[a] : (int)fl);
        lo[a] = clampi(c, 0, N[a] - 1);
        hi[a] = clampi(c + 1, 0, N[a] - 1);
    }
    double acc = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
        int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        double w = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);
        acc += w * voxel(v, bx ? hi[0] : lo[0], by ? hi[1] : lo[1], bz ? hi[2] : lo[2]);
    }
    return acc;
}

/* Transfer function: M entries evenly spaced over [vmin, vmax], linear
   interpolation, clamped at both ends. */
static void tf_lookup(const orc_tf* tf, double v, double out[4]) {
    double x = (v - (double)tf->vmin) / ((double)tf->vmax - (double)tf->vmin) * (double)(tf->M - 1);
    if (x < 0.0) x = 0.0;
    if (x > (double)(tf->M - 1)) x = (double)(tf->M - 1);
    int i = (int)floor(x);
    if (i > tf->M - 2) i = tf->M - 2;
    double f = x - (double)i;
    for (int ch = 0; ch < 4; ++ch)
        out[ch] = (1.0 - f) * (double)tf->rgba[4 * i + ch] + f * (double)tf->rgba[4 * (i + 1) + ch];
}

static int valid_inputs(const orc_volume* vol, const orc_tf* tf) {
    if (!vol || !tf || !vol->data || !tf->rgba) return 0;
    if (vol->dtype != ORC_U8 && vol->dtype != ORC_U16) return 0;
    if (vol->nx < 1 || vol->ny < 1 || vol->nz < 1) return 0;
    if (tf->M < 2 || !(tf->vmax > tf->vmin)) return 0;
    return 1;
}

static int vol_nmax(const orc_volume* v) {
    int m = v->nx;
    if (v->ny > m) m = v->ny;
    if (v->nz > m) m = v->nz;
    return m;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: the illumination attenuation buffer, slice by slice.   */
/*
 * B[k][j][i] holds the light arriving at slice k: B_0 = 1 and
 * B_k = prod_{j<k} (1 - alpha_j), alpha_j the transfer-function opacity at the
 * texel's point on slice j (back-to-front blending of Eq. 4 applied to a
 * scalar transmittance).  Texels whose point lies outside the unit cube see no
 * medium (alpha = 0).
 */

typedef struct {
    const orc_volume* vol;
    const orc_tf* tf;
    const orc_light* lt;
    const orc_build_opts* opt;
    double* T;
    double* Bk;
    float sk;
    double spacing_vox;
    int j0;
} sweep_ctx;

static void sweep_rows(void* p, long lo, long hi) {
    sweep_ctx* s = (sweep_ctx*)p;
    const int R = s->lt->R;
    for (long j = s->j0 + lo; j < s->j0 + hi; ++j) {
        for (int i = 0; i < R; ++i) {
            size_t t = (size_t)j * (size_t)R + (size_t)i;
            float P[3];
            texel_world(s->lt, i, (int)j, s->sk, P);
            double alpha = 0.0;
            if (P[0] >= 0.0f && P[0] <= 1.0f && P[1] >= 0.0f && P[1] <= 1.0f &&
                P[2] >= 0.0f && P[2] <= 1.0f) {
                int cell[3];
                double rgba[4];
                tf_lookup(s->tf, sample_volume(s->vol, P, cell), rgba);
                alpha = rgba[3];
                if (s->opt && s->opt->opacity_correction)
                    alpha = 1.0 - pow(1.0 - alpha, s->spacing_vox * column_stretch(s->lt, i, (int)j));
            }
            const int depth = s->opt && s->opt->quantity == ORC_OPTICAL_DEPTH;
            double stored = s->T[t];
            if (s->opt && s->opt->comp_n != 0.0f) {
                /* Darkening compensation: scale the slice by (1 + alpha)^n
                   (in depth form: subtract n ln(1 + alpha)). */
                if (depth) {
                    stored = stored - (double)s->opt->comp_n * log1p(alpha);
                    if (stored < 0.0) stored = 0.0;
                } else {
                    stored = stored * pow(1.0 + alpha, (double)s->opt->comp_n);
                    if (stored > 1.0) stored = 1.0;
                }
            }
            s->Bk[t] = stored;
            if (depth) {
                /* Eq. 5-6: extinctions add; tau = -ln(1 - alpha). */
                double D = s->T[t] + (-log1p(-alpha));
                s->T[t] = D < ORC_DEPTH_MAX ? D : ORC_DEPTH_MAX;
            } else {
                s->T[t] = s->T[t] * (1.0 - alpha);
            }
        }
    }
}

/* Texel rows [j0, j1) of every slice (the rest of B is left untouched); the
   CPU-baseline timing runs a band of rows. */
int orc_build_stack_rows(const orc_volume* vol, const orc_tf* tf, const orc_light* lt,
                         const orc_build_opts* opt, int j0, int j1, double* B) {
    if (!valid_inputs(vol, tf) || !lt || !B || lt->n < 1 || lt->R < 1) return ORC_EINVAL;
    if (j0 < 0 || j1 > lt->R || j0 >= j1) return ORC_EINVAL;
    const size_t RR = (size_t)lt->R * (size_t)lt->R;
    double* T = (double*)malloc(RR * sizeof(double));
    if (!T) return ORC_ENOMEM;
    if (opt && opt->quantity != ORC_TRANSMITTANCE && opt->quantity != ORC_OPTICAL_DEPTH) {
        free(T);
        return ORC_EINVAL;
    }
    /* LightBuffer initialised to full light: T = 1, or optical depth 0. */
    const double full = (opt && opt->quantity == ORC_OPTICAL_DEPTH) ? 0.0 : 1.0;
    for (size_t t = 0; t < RR; ++t) T[t] = full;
    sweep_ctx s;
    s.vol = vol;
    s.tf = tf;
    s.lt = lt;
    s.opt = opt;
    s.T = T;
    s.spacing_vox = (double)lt->dL * (double)vol_nmax(vol);
    s.j0 = j0;
    /* For each slice, nearest to the light first: evaluate, store, blend. */
    for (int k = 0; k < lt->n; ++k) {
        s.sk = slice_offset(lt, k);
        s.Bk = B + (size_t)k * RR;
        parallel_for(j1 - j0, 4, sweep_rows, &s);
    }
    free(T);
    return ORC_OK;
}

int orc_build_stack(const orc_volume* vol, const orc_tf* tf, const orc_light* lt,
                    const orc_build_opts* opt, double* B) {
    if (!lt) return ORC_EINVAL;
    return orc_build_stack_rows(vol, tf, lt, opt, 0, lt->R, B);
}

/* ------------------------------------------------------------------ */
/* Camera and eye rays (index path).                                   */

int orc_frame_setup(const orc_camera* cam, int W, int H, float step_vox, int Nmax, orc_frame* fr) {
    if (!cam || !fr || W < 1 || H < 1 || Nmax < 1 || !(step_vox > 0.0f)) return ORC_EINVAL;
    memset(fr, 0, sizeof(*fr));
    float fw[3], r0[3];
    for (int a = 0; a < 3; ++a) fw[a] = cam->target[a] - cam->eye[a];
    float nf = sqrtf(dot3f(fw, fw));
    if (!(nf > 0.0f) || !isfinite(nf)) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a) fr->f[a] = fw[a] / nf;
    cross3f(fr->f, cam->up, r0);
    float nr = sqrtf(dot3f(r0, r0));
    if (!(nr > 0.0f) || !isfinite(nr)) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a) fr->r[a] = r0[a] / nr;
    cross3f(fr->r, fr->f, fr->u);
    for (int a = 0; a < 3; ++a) fr->eye[a] = cam->eye[a];
    float aspect = (float)W / (float)H;
    if (cam->perspective) {
        if (!(cam->fovy_deg > 0.0f && cam->fovy_deg < 180.0f)) return ORC_EINVAL;
        float th = (float)tan((double)cam->fovy_deg * (M_PI / 360.0));
        fr->sx = th * aspect;
        fr->sy = th;
    } else {
        if (!(cam->ortho_half_height > 0.0f)) return ORC_EINVAL;
        fr->sx = cam->ortho_half_height * aspect;
        fr->sy = cam->ortho_half_height;
    }
    fr->dt = step_vox / (float)Nmax;
    fr->perspective = cam->perspective ? 1 : 0;
    fr->W = W;
    fr->H = H;
    fr->Nmax = Nmax;
    return ORC_OK;
}

/* Light-space coordinates (lambda, tu, tv) of a world point (Eq. 9, Eq. 10).
   Directional: lambda = kappa (L.X - min), tu = sigma (X - c).U + rho0, tv
   likewise.  Point light: with e = X - P and depth d = e.L, lambda =
   kappa (d - min), tu = sigma (e.U / d) + rho0, tv likewise (the perspective
   divide; a depth below 1e-6 -- at or behind the light -- counts as 1e-6). */
static void light_coords(const orc_light* lt, const float X[3], float out[3]) {
    if (lt->point) {
        float e[3] = {X[0] - lt->P[0], X[1] - lt->P[1], X[2] - lt->P[2]};
        float d = dot3f(e, lt->L);
        out[0] = (d - lt->min) * lt->kappa;
        float ds = d > 1e-6f ? d : 1e-6f;
        float su = dot3f(e, lt->U) / ds;
        float sv = dot3f(e, lt->V) / ds;
        out[1] = fmaf(su, lt->sigma, lt->rho0);
        out[2] = fmaf(sv, lt->sigma, lt->rho0);
        return;
    }
    float LX = dot3f(lt->L, X);
    float dl = LX - lt->min;
    out[0] = dl * lt->kappa;
    float xc[3] = {X[0] - 0.5f, X[1] - 0.5f, X[2] - 0.5f};
    out[1] = fmaf(dot3f(xc, lt->U), lt->sigma, lt->rho0);
    out[2] = fmaf(dot3f(xc, lt->V), lt->sigma, lt->rho0);
}

int orc_light_coords(const orc_light* lt, const float X[3], float out[3]) {
    if (!lt || !X || !out) return ORC_EINVAL;
    light_coords(lt, X, out);
    return ORC_OK;
}

/* World positions of a sample's scattering points under a point light
   (Section 3.2.3 with the light direction taken at the sample):
   shell q: S +- q r e_a; cone: w = (S - P)/|S - P| the direction the light
   travels at S, ring n (1, 2) centred at S - n dL w with radius n dL tan(phi),
   its four points B_proj turned by m pi/2 about w (Eq. 11: w x B for a
   quarter turn), B_proj the unit part of -d (towards the eye) orthogonal to w
   (U's part if that is below 1e-6).  Returns the number of points. */
static int point_neighbours(const orc_light* lt, const orc_render_opts* ro, int Nmax,
                            const float S[3], const float d[3], float X[ORC_MAX_NB][3]) {
    if (ro->mode == ORC_SHELL) {
        const int Q = ro->shell_count > 0 ? ro->shell_count : 1;
        for (int q = 1; q <= Q; ++q) {
            float r = ((float)q * ro->shell_radius_vox) / (float)Nmax;
            for (int a = 0; a < 3; ++a)
                for (int sgn = 0; sgn < 2; ++sgn) {
                    float* o = X[6 * (q - 1) + 2 * a + sgn];
                    o[0] = S[0];
                    o[1] = S[1];
                    o[2] = S[2];
                    o[a] = sgn ? S[a] - r : S[a] + r;
                }
        }
        return 6 * Q;
    }
    if (ro->mode != ORC_CONE) return 0;
    float e[3] = {S[0] - lt->P[0], S[1] - lt->P[1], S[2] - lt->P[2]};
    float le = sqrtf(dot3f(e, e));
    float w[3] = {e[0] / le, e[1] / le, e[2] / le};
    float md[3] = {-d[0], -d[1], -d[2]};
    float pr = dot3f(md, w);
    float b[3];
    for (int a = 0; a < 3; ++a) b[a] = fmaf(-pr, w[a], md[a]);
    float nb = sqrtf(dot3f(b, b));
    if (!(nb >= 1e-6f)) {
        pr = dot3f(lt->U, w);
        for (int a = 0; a < 3; ++a) b[a] = fmaf(-pr, w[a], lt->U[a]);
        nb = sqrtf(dot3f(b, b));
    }
    float B[4][3];
    for (int a = 0; a < 3; ++a) B[0][a] = b[a] / nb;
    cross3f(w, B[0], B[1]);
    for (int a = 0; a < 3; ++a) {
        B[2][a] = -B[0][a];
        B[3][a] = -B[1][a];
    }
    float tanphi = (float)tan((double)ro->cone_half_angle_deg * (M_PI / 180.0));
    for (int ring = 1; ring <= 2; ++ring) {
        float dist = (float)ring * lt->dL;
        float rad = dist * tanphi;
        float c[3];
        for (int a = 0; a < 3; ++a) c[a] = fmaf(-dist, w[a], S[a]);
        for (int m = 0; m < 4; ++m)
            for (int a = 0; a < 3; ++a) X[(ring - 1) * 4 + m][a] = fmaf(rad, B[m][a], c[a]);
    }
    return 8;
}

int orc_point_neighbours(const orc_light* lt, const orc_render_opts* ro, int Nmax,
                         const float S[3], const float d[3], float* X) {
    if (!lt || !ro || !S || !d || !X || !lt->point) return -1;
    return point_neighbours(lt, ro, Nmax, S, d, (float(*)[3])X);
}

/* Rotation by theta_m = m pi/2 about L of a unit vector in the light plane,
   written in the (U, V) frame where L x U = V and L x V = -U (Eq. 11 with
   cos/sin of quarter turns and L . B = 0). */
static void quarter_turn(int m, float bu, float bv, float* cu, float* cv) {
    switch (m & 3) {
        case 0: *cu = bu; *cv = bv; break;
        case 1: *cu = -bv; *cv = bu; break;
        case 2: *cu = -bu; *cv = -bv; break;
        default: *cu = bv; *cv = -bu; break;
    }
}

int orc_ray_setup(const orc_light* lt, const orc_frame* fr, const orc_render_opts* ro,
                  int x, int y, orc_ray* ray) {
    if (!lt || !fr || !ro || !ray) return ORC_EINVAL;
    if (ro->shell_count < 0 || ro->shell_count > ORC_MAX_SHELLS) return ORC_EINVAL;
    memset(ray, 0, sizeof(*ray));
    /* Pixel centre (x + 1/2, y + 1/2); row 0 at the top. */
    float qx = (float)(2 * x + 1) / (float)fr->W;
    float qy = (float)(2 * y + 1) / (float)fr->H;
    float px = (qx - 1.0f) * fr->sx;
    float py = (1.0f - qy) * fr->sy;
    if (fr->perspective) {
        float dw[3];
        for (int a = 0; a < 3; ++a) dw[a] = fmaf(py, fr->u[a], fmaf(px, fr->r[a], fr->f[a]));
        float nd = sqrtf(dot3f(dw, dw));
        for (int a = 0; a < 3; ++a) {
            ray->o[a] = fr->eye[a];
            ray->d[a] = dw[a] / nd;
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            ray->o[a] = fmaf(py, fr->u[a], fmaf(px, fr->r[a], fr->eye[a]));
            ray->d[a] = fr->f[a];
        }
    }
    /* Slab intersection with [0,1]^3; samples start no earlier than t = 0. */
    float t0 = 0.0f, t1 = INFINITY;
    int hit = 1;
    for (int a = 0; a < 3; ++a) {
        if (ray->d[a] != 0.0f) {
            float ta = (0.0f - ray->o[a]) / ray->d[a];
            float tb = (1.0f - ray->o[a]) / ray->d[a];
            float tn = fminf(ta, tb), tx = fmaxf(ta, tb);
            if (tn > t0) t0 = tn;
            if (tx < t1) t1 = tx;
        } else if (ray->o[a] < 0.0f || ray->o[a] > 1.0f) {
            hit = 0;
        }
    }
    ray->t0 = t0;
    ray->t1 = t1;
    ray->hit = hit && (t0 < t1);

    /* Light-space coordinates are affine in t: l(t) = lo + t ld. */
    float LO = dot3f(lt->L, ray->o);
    float dl = LO - lt->min;
    ray->lo[0] = dl * lt->kappa;
    ray->ld[0] = dot3f(lt->L, ray->d) * lt->kappa;
    float oc[3] = {ray->o[0] - 0.5f, ray->o[1] - 0.5f, ray->o[2] - 0.5f};
    ray->lo[1] = fmaf(dot3f(oc, lt->U), lt->sigma, lt->rho0);
    ray->ld[1] = dot3f(ray->d, lt->U) * lt->sigma;
    ray->lo[2] = fmaf(dot3f(oc, lt->V), lt->sigma, lt->rho0);
    ray->ld[2] = dot3f(ray->d, lt->V) * lt->sigma;

    if (ro->mode == ORC_SHELL) {
        /* Shells (Section 3.2.3): shell q = 1..Q holds the six points
           S +- q r e_a, r = shell_radius_vox voxels. */
        const int Q = ro->shell_count > 0 ? ro->shell_count : 1;
        ray->nnb = 6 * Q;
        for (int q = 1; q <= Q; ++q) {
            float r = ((float)q * ro->shell_radius_vox) / (float)fr->Nmax;
            for (int a = 0; a < 3; ++a) {
                float rl = r * lt->L[a];
                float ru = r * lt->U[a];
                float rv = r * lt->V[a];
                float off[3] = {rl * lt->kappa, ru * lt->sigma, rv * lt->sigma};
                for (int s = 0; s < 2; ++s)
                    for (int c = 0; c < 3; ++c)
                        ray->nb[6 * (q - 1) + 2 * a + s][c] = s ? -off[c] : off[c];
            }
        }
    } else if (ro->mode == ORC_CONE) {
        /* Cone: apex S, axis towards the light.  Ring n (n = 1, 2) is centred
           at c_n = S - n dL L with radius n dL tan(phi); its four points are
           B_proj rotated by m pi/2 about L (Eq. 11).  B_proj is the unit
           part of E - S orthogonal to L; along an eye ray E - S is parallel
           to -d, so B_proj is fixed per ray. */
        float bu0 = -ray->ld[1];
        float bv0 = -ray->ld[2];
        float pu = bu0 * bu0;
        float pv = bv0 * bv0;
        float nb = sqrtf(pu + pv);
        float thr = 1e-6f * lt->sigma;
        float bu = 1.0f, bv = 0.0f; /* view parallel to the light: use U */
        if (nb >= thr) {
            bu = bu0 / nb;
            bv = bv0 / nb;
        }
        float tanphi = (float)tan((double)ro->cone_half_angle_deg * (M_PI / 180.0));
        ray->nnb = 8;
        for (int ring = 1; ring <= 2; ++ring) {
            float dist = (float)ring * lt->dL;
            float radw = dist * tanphi;
            float rad = radw * lt->sigma;
            for (int m = 0; m < 4; ++m) {
                float cu, cv;
                quarter_turn(m, bu, bv, &cu, &cv);
                float* o = ray->nb[(ring - 1) * 4 + m];
                o[0] = -(float)ring; /* n slice spacings towards the light */
                o[1] = rad * cu;
                o[2] = rad * cv;
            }
        }
    }
    return ORC_OK;
}

/* Bilinear lookup in slice k of the buffer (Eq. 9 for k, Eq. 10 for UV):
   k = clamp(floor(lambda + 1/2), 0, n - 1); texel centres at integer (tu, tv),
   clamp to edge. */
static double bilinear_slice(const double* B, const orc_light* lt, int k, float tu, float tv,
                             int* rec) {
    const int R = lt->R;
    int iu = floor_clamp(tu, -1, R);
    int iv = floor_clamp(tv, -1, R);
    if (rec) {
        rec[0] = k;
        rec[1] = iu;
        rec[2] = iv;
    }
    if (!B) return 1.0;
    double fu = (double)tu - floor((double)tu);
    double fv = (double)tv - floor((double)tv);
    int i0 = clampi(iu, 0, R - 1), i1 = clampi(iu + 1, 0, R - 1);
    int j0 = clampi(iv, 0, R - 1), j1 = clampi(iv + 1, 0, R - 1);
    const double* S = B + (size_t)k * (size_t)R * (size_t)R;
    double top = (1.0 - fu) * S[(size_t)j0 * R + i0] + fu * S[(size_t)j0 * R + i1];
    double bot = (1.0 - fu) * S[(size_t)j1 * R + i0] + fu * S[(size_t)j1 * R + i1];
    return (1.0 - fv) * top + fv * bot;
}

static double stack_lookup(const double* B, const orc_light* lt, float lam, float tu, float tv,
                           int* rec) {
    float lh = lam + 0.5f;
    int k = floor_clamp(lh, 0, lt->n - 1);
    return bilinear_slice(B, lt, k, tu, tv, rec);
}

/* Light factor of one lookup point: the buffer value at (lambda, tu, tv),
   from the nearest slice (as stack_lookup) or, with linear slice filtering,
   interpolated between slices k0 = clamp(floor(lambda), 0, n - 1) and
   min(k0 + 1, n - 1) with weight lambda - k0 clamped to [0, 1]; then, for an
   optical-depth buffer, the transmittance exp(-D) (Eq. 5-6). */
static double light_lookup(const double* B, const orc_light* lt, const orc_render_opts* ro,
                           float lam, float tu, float tv, int* rec) {
    double v;
    if (ro->slice_filter == ORC_SLICE_LINEAR) {
        int k0 = floor_clamp(lam, 0, lt->n - 1);
        int k1 = k0 + 1 < lt->n ? k0 + 1 : k0;
        double w = (double)lam - (double)k0;
        if (w < 0.0) w = 0.0;
        if (w > 1.0) w = 1.0;
        double b0 = bilinear_slice(B, lt, k0, tu, tv, rec);
        double b1 = bilinear_slice(B, lt, k1, tu, tv, NULL);
        v = (1.0 - w) * b0 + w * b1;
    } else {
        v = stack_lookup(B, lt, lam, tu, tv, rec);
    }
    if (!B) return 1.0;
    return ro->quantity == ORC_OPTICAL_DEPTH ? exp(-v) : v;
}

/* ------------------------------------------------------------------ */
/* The eye pass: one ray per pixel, front-to-back compositing.         */

typedef struct {
    const orc_volume* vol;
    const orc_tf* tf;
    const orc_light* lt;
    const double* B;
    const orc_frame* fr;
    const orc_render_opts* ro;
    const int* xs;
    const int* ys;
    double* out;
    double* alt;
    uint8_t* ambiguous;
    long long* nsamples;
    long long* nsamples_alt;
    double* end;
    long long* nsamples_end;
    int32_t* trace;
    int trace_max;
    int* trace_count;
} march_ctx;

static void march_one(const march_ctx* s, long p) {
    const orc_render_opts* ro = s->ro;
    const int x = s->xs[p], y = s->ys[p];
    orc_ray ray;
    orc_ray_setup(s->lt, s->fr, ro, x, y, &ray);
    double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
    long long count = 0;
    int ntrace = 0;
    /* Early ray termination (Eq. 3; the test A > ert after each composited
       sample, reading R12).  A binary32 renderer carries A with an error far
       below ert_band, so where the binary64 A passes within ert_band of ert
       it may stop at any sample of a window: from lo, the first sample with
       A > ert - band, to hi, the first with A > ert + band (or the ray's last
       sample if none).  "out" is the binary64 decision: the first sample with
       A > ert, else the ray's end.  "alt" is the state at the window's other
       end (lo, unless out is at lo; then hi).  ambiguous = 0 for a window of
       one sample (one outcome), 1 for two samples (out and alt are both
       outcomes), 2 for three or more (out and alt are its two ends and the
       binary64 decision; the samples between them are outcomes too). */
    const double ert = (double)ro->ert, band = ro->ert_band;
    double LC[3] = {0, 0, 0}, LA = 0.0, MC[3] = {0, 0, 0}, MA = 0.0;
    long long lo_at = -1, main_at = -1, last = -1, Lcount = 0, Mcount = 0;
    if (ray.hit) {
        for (long i = 0;; ++i) {
            /* Sample i at t_i = t0 + i dt while t_i < t1. */
            float t = fmaf((float)i, s->fr->dt, ray.t0);
            if (!(t < ray.t1)) break;
            float S[3];
            for (int a = 0; a < 3; ++a) S[a] = fmaf(t, ray.d[a], ray.o[a]);
            float l[3];
            if (s->lt->point)
                light_coords(s->lt, S, l); /* perspective: per sample */
            else
                for (int c = 0; c < 3; ++c) l[c] = fmaf(t, ray.ld[c], ray.lo[c]);
            int cell[3];
            double rgba[4];
            tf_lookup(s->tf, sample_volume(s->vol, S, cell), rgba);
            double alpha = rgba[3];
            if (ro->opacity_correction) alpha = 1.0 - pow(1.0 - alpha, (double)ro->step_vox);

            int32_t* rec = NULL;
            if (s->trace && ntrace < s->trace_max) {
                rec = s->trace + (size_t)ntrace * ORC_TRACE_WORDS;
                for (int w = 0; w < ORC_TRACE_WORDS; ++w) rec[w] = ORC_TRACE_NONE;
                rec[0] = (int32_t)i;
                memcpy(&rec[1], &t, 4);
                memcpy(&rec[2], &l[0], 4);
                memcpy(&rec[3], &l[1], 4);
                memcpy(&rec[4], &l[2], 4);
                rec[5] = cell[0];
                rec[6] = cell[1];
                rec[7] = cell[2];
                rec[35] = ray.nnb;
                ++ntrace;
            }

            /* Attenuation coefficient a_s of the sample (Eq. 7). */
            double coef = 1.0;
            if (ro->mode == ORC_SHADOW) {
                coef = light_lookup(s->B, s->lt, ro, l[0], l[1], l[2], rec ? rec + 8 : NULL);
            } else {
                if (rec) light_lookup(NULL, s->lt, ro, l[0], l[1], l[2], rec + 8);
                if (ro->mode == ORC_SHELL || ro->mode == ORC_CONE) {
                    double sum = 0.0;
                    float X[ORC_MAX_NB][3];
                    int nnb = ray.nnb;
                    if (s->lt->point) nnb = point_neighbours(s->lt, ro, s->fr->Nmax, S, ray.d, X);
                    for (int j = 0; j < nnb; ++j) {
                        float q[3];
                        if (s->lt->point) {
                            light_coords(s->lt, X[j], q);
                        } else {
                            q[0] = l[0] + ray.nb[j][0];
                            q[1] = l[1] + ray.nb[j][1];
                            q[2] = l[2] + ray.nb[j][2];
                        }
                        /* The record has room for the first 8 neighbours. */
                        int* nrec = (rec && j < 8) ? rec + 11 + 3 * j : NULL;
                        sum += light_lookup(s->B, s->lt, ro, q[0], q[1], q[2], nrec);
                    }
                    coef = sum / (double)nnb;
                }
            }
            double lf = (double)ro->ambient + (1.0 - (double)ro->ambient) * coef;

            /* Eq. 3, front to back, with opacity-weighted colour (Eq. 2). */
            for (int ch = 0; ch < 3; ++ch) {
                double csrc = lf * (double)ro->color[ch] * alpha * rgba[ch];
                C[ch] = C[ch] + (1.0 - A) * csrc;
            }
            A = A + (1.0 - A) * alpha;
            ++count;
            last = (long long)i;

            /* Early ray termination: the window's start, the binary64
               decision, and its end (where the loop stops). */
            if (lo_at < 0 && A > ert - band) {
                lo_at = (long long)i;
                LC[0] = C[0]; LC[1] = C[1]; LC[2] = C[2]; LA = A; Lcount = count;
            }
            if (main_at < 0 && A > ert) {
                main_at = (long long)i;
                MC[0] = C[0]; MC[1] = C[1]; MC[2] = C[2]; MA = A; Mcount = count;
            }
            if (A > ert + band) break;
        }
    }
    /* Here C, A, count hold the state at the window's end (hi) or the ray's end. */
    double outC[3], outA, altC[3], altA;
    long long outcount = count, altcount = count;
    int amb = 0;
    for (int ch = 0; ch < 3; ++ch) outC[ch] = altC[ch] = C[ch];
    outA = altA = A;
    if (main_at >= 0) {
        for (int ch = 0; ch < 3; ++ch) outC[ch] = MC[ch];
        outA = MA;
        outcount = Mcount;
    }
    if (lo_at >= 0 && lo_at < last) {
        amb = last - lo_at >= 2 ? 2 : 1;
        if (main_at != lo_at) {
            for (int ch = 0; ch < 3; ++ch) altC[ch] = LC[ch];
            altA = LA;
            altcount = Lcount;
        }
    }
    /* Background behind the remaining transparency. */
    double* o = s->out + 4 * (size_t)p;
    for (int ch = 0; ch < 3; ++ch) o[ch] = outC[ch] + (1.0 - outA) * (double)ro->bg[ch];
    o[3] = outA + (1.0 - outA) * (double)ro->bg[3];
    if (s->alt) {
        double* q = s->alt + 4 * (size_t)p;
        for (int ch = 0; ch < 3; ++ch) q[ch] = altC[ch] + (1.0 - altA) * (double)ro->bg[ch];
        q[3] = altA + (1.0 - altA) * (double)ro->bg[3];
    }
    if (s->ambiguous) s->ambiguous[p] = (uint8_t)amb;
    if (s->nsamples) s->nsamples[p] = outcount;
    if (s->nsamples_alt) s->nsamples_alt[p] = altcount;
    if (s->end) {
        double* q = s->end + 4 * (size_t)p;
        for (int ch = 0; ch < 3; ++ch) q[ch] = C[ch] + (1.0 - A) * (double)ro->bg[ch];
        q[3] = A + (1.0 - A) * (double)ro->bg[3];
    }
    if (s->nsamples_end) s->nsamples_end[p] = count;
    if (s->trace_count) *s->trace_count = ntrace;
}

static void march_range(void* p, long lo, long hi) {
    const march_ctx* s = (const march_ctx*)p;
    for (long q = lo; q < hi; ++q) march_one(s, q);
}

static int render_common(const orc_volume* vol, const orc_tf* tf, const orc_light* lt,
                         const double* B, const orc_camera* cam, int W, int H,
                         const orc_render_opts* ro, const int* xs, const int* ys, long count,
                         double* out, double* alt, uint8_t* ambiguous, long long* nsamples,
                         long long* nsamples_alt, double* end, long long* nsamples_end,
                         int32_t* trace, int trace_max, int* trace_count) {
    if (!valid_inputs(vol, tf) || !lt || !cam || !ro || !out || !xs || !ys) return ORC_EINVAL;
    if (ro->mode < ORC_NONE || ro->mode > ORC_CONE) return ORC_EINVAL;
    if (ro->mode != ORC_NONE && !B) return ORC_EINVAL;
    if (ro->quantity != ORC_TRANSMITTANCE && ro->quantity != ORC_OPTICAL_DEPTH) return ORC_EINVAL;
    if (ro->slice_filter != ORC_SLICE_NEAREST && ro->slice_filter != ORC_SLICE_LINEAR)
        return ORC_EINVAL;
    if (ro->shell_count < 0 || ro->shell_count > ORC_MAX_SHELLS) return ORC_EINVAL;
    orc_frame fr;
    int rc = orc_frame_setup(cam, W, H, ro->step_vox, vol_nmax(vol), &fr);
    if (rc) return rc;
    for (long p = 0; p < count; ++p)
        if (xs[p] < 0 || xs[p] >= W || ys[p] < 0 || ys[p] >= H) return ORC_EINVAL;
    march_ctx s;
    s.vol = vol;
    s.tf = tf;
    s.lt = lt;
    s.B = B;
    s.fr = &fr;
    s.ro = ro;
    s.xs = xs;
    s.ys = ys;
    s.out = out;
    s.alt = alt;
    s.ambiguous = ambiguous;
    s.nsamples = nsamples;
    s.nsamples_alt = nsamples_alt;
    s.end = end;
    s.nsamples_end = nsamples_end;
    s.trace = trace;
    s.trace_max = trace_max;
    s.trace_count = trace_count;
    if (trace) {
        march_range(&s, 0, count);
    } else {
        parallel_for(count, 64, march_range, &s);
    }
    return ORC_OK;
}

/* Render the listed pixels of a W x H image.  out, alt, end: count x RGBA
   (binary64); alt differs from out only on ERT-ambiguous pixels (ambiguous
   1 or 2, see march_one); end is the state at the end of the ERT window (out
   where there is no window).  nsamples, nsamples_alt, nsamples_end: the
   samples composited for each.  alt, end and their counts may be NULL. */
int orc_render_pixels(const orc_volume* vol, const orc_tf* tf, const orc_light* lt,
                      const double* B, const orc_camera* cam, int W, int H,
                      const orc_render_opts* ro, const int* xs, const int* ys, long count,
                      double* out, double* alt, uint8_t* ambiguous, long long* nsamples,
                      long long* nsamples_alt, double* end, long long* nsamples_end) {
    return render_common(vol, tf, lt, B, cam, W, H, ro, xs, ys, count, out, alt, ambiguous,
                         nsamples, nsamples_alt, end, nsamples_end, NULL, 0, NULL);
}

/* Per-sample index-path record of one pixel's ray (ORC_TRACE_WORDS int32 per
   sample): i, t, lambda, tu, tv (binary32 bits), voxel cell (3), the sample's
   own lookup cell (k, iu, iv), 8 neighbour cells (k, iu, iv), neighbour count. */
int orc_trace_pixel(const orc_volume* vol, const orc_tf* tf, const orc_light* lt,
                    const double* B, const orc_camera* cam, int W, int H,
                    const orc_render_opts* ro, int x, int y, int32_t* rec, int max_rec,
                    int* n_rec) {
    if (!rec || max_rec < 0 || !n_rec) return ORC_EINVAL;
    double out[4];
    *n_rec = 0;
    return render_common(vol, tf, lt, B, cam, W, H, ro, &x, &y, 1, out, NULL, NULL, NULL, NULL,
                         NULL, NULL, rec, max_rec, n_rec);
}

/* ------------------------------------------------------------------ */
/* Eq. 1 along the light ray, absorption only: the exact transmittance  */
/* exp(-integral of kappa) from where the light enters the cube to P,   */
/* kappa = -ln(1 - alpha) per voxel of path (the extinction whose       */
/* one-voxel step gives opacity alpha).  Composite Simpson, m steps.    */

double orc_transmittance_bruteforce(const orc_volume* vol, const orc_tf* tf, const double L[3],
                                    const double P[3], long m) {
    if (!valid_inputs(vol, tf) || !L || !P || m < 2) return NAN;
    if (m & 1) ++m;
    /* Walk back towards the light: X(s) = P - s L, s in [0, s_exit]. */
    double s_exit = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (L[a] > 0.0) {
            double s = P[a] / L[a];
            if (s < s_exit) s_exit = s;
        } else if (L[a] < 0.0) {
            double s = (P[a] - 1.0) / L[a];
            if (s < s_exit) s_exit = s;
        }
    }
    if (!(s_exit > 0.0)) return 1.0;
    const double nvox = (double)vol_nmax(vol);
    const double h = s_exit / (double)m;
    double sum = 0.0;
    for (long q = 0; q <= m; ++q) {
        double s = h * (double)q;
        double X[3] = {P[0] - s * L[0], P[1] - s * L[1], P[2] - s * L[2]};
        double rgba[4];
        tf_lookup(tf, sample_volume_f64(vol, X), rgba);
        double kap = -log(1.0 - rgba[3]) * nvox;
        double w = (q == 0 || q == m) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
        sum += w * kap;
    }
    return exp(-sum * h / 3.0);
}

/* Exported single-step helpers, so tests can pin each stage on its own. */
double orc_sample_volume(const orc_volume* vol, const float P[3], int cell[3]) {
    int tmp[3];
    return sample_volume(vol, P, cell ? cell : tmp);
}

void orc_tf_lookup(const orc_tf* tf, double v, double out[4]) { tf_lookup(tf, v, out); }

int orc_texel_world(const orc_light* lt, int i, int j, int k, float P[3]) {
    if (!lt || !P) return ORC_EINVAL;
    texel_world(lt, i, j, slice_offset(lt, k), P);
    return ORC_OK;
}

double orc_stack_lookup(const double* B, const orc_light* lt, float lam, float tu, float tv,
                        int rec[3]) {
    return stack_lookup(B, lt, lam, tu, tv, rec);
}

double orc_light_lookup(const double* B, const orc_light* lt, const orc_render_opts* ro,
                        float lam, float tu, float tv, int rec[3]) {
    return light_lookup(B, lt, ro, lam, tu, tv, rec);
}
