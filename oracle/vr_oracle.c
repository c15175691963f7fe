/*
 * vr_oracle.c -- plain, slow CPU reference of the bricked ray-casting method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * bench load this library.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes follows Hassan, Fluke & Barnes, "Interactive Visualization of the Largest
 * Radioastronomy Cubes":
 *   Section 2 (ray casting): each pixel's ray is traced through the cube; a transfer function
 *       maps each sample value to colour and opacity; colour and opacity are accumulated.
 *   Section 2.4 (ray-casting process): ray/box test gives entry and exit; early ray termination
 *       stops a ray once its accumulated opacity reaches its maximum; MIP mode returns the
 *       maximum sampled scalar per pixel.
 *   Section 2.5 (image composition): sub-images are blended with the associative "over"
 *       operator, so partial images of sub-volumes compose to the whole-volume image.
 *
 * The oracle is the unbricked definition: one ray per pixel over the whole cube, samples on
 * the lattice t_k = k*step measured from the ray origin, trilinear interpolation of the
 * voxel-centred field with clamp-to-edge, a piecewise-linear RGBA table, front-to-back "over"
 * in FP64.  Readings where the paper is silent:
 *   - Decisions that pick integers (which lattice samples lie in the cube, and which brick owns
 *     a sample) are taken in FP32 with IEEE operations in a fixed order (ray generation, slab
 *     t-values, ceil(t/step)), the same order the renderer states.  Sample positions, values,
 *     colours and compositing are FP64.
 *   - Early ray termination is per brick segment when a brick size is given (each brick's
 *     segment of the ray stops on its own opacity, the way a sort-last renderer can apply it),
 *     and global otherwise.  The test is T <= 1 - tau after compositing a sample.
 *   - MIP of a pixel with no samples reports vmin.
 *   - FP16 / BF16 bricks: each brick's stored region (core plus ghost) is scaled by a power of
 *     two chosen from its max |v|, then rounded to nearest-even; a sample reads the voxels as
 *     stored in the brick that owns it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    const float *vox;               /* [z][y][x], x fastest */
    int64_t nx, ny, nz;
    const float *lut;               /* nlut x 4 RGBA, non-premultiplied */
    int32_t nlut;
    float vmin, vmax;
    float view[16];                 /* world -> eye, row-major */
    int32_t proj;                   /* 0 orthographic, 1 perspective */
    float param;                    /* ortho: image height (world units); persp: vertical fov (rad) */
    int32_t W, H;
    int32_t mode;                   /* 0 DVR, 1 MIP (FP64), 2 MIP in the FP32 operation order */
    float step, tau;
    int64_t bx, by, bz;             /* brick core size; 0 = one segment per ray */
    int32_t quant;                  /* 0 FP32 voxels, 1 FP16 bricks, 2 BF16 bricks */
    int32_t ghost;                  /* ghost width of the stored brick region */
    int32_t nthreads;
    int32_t procedural;             /* 1: voxels come from the procedural cube (vox unused) */
    uint64_t proc_seed;
    const uint8_t *channels;        /* per spectral channel z: 0 = disabled (NULL: all enabled) */
    int64_t win_lo[3], win_hi[3];   /* render window [lo, hi) in voxels (hi <= lo: whole cube) */
    int32_t term_global;            /* DVR early termination: 0 per brick segment, 1 whole ray */
    uint64_t *sig;                  /* DVR, optional (NULL: none): per listed pixel, a hash of its
                                       piecewise structure -- for every composited sample, the
                                       table interval or the clamp side its value falls in, and
                                       the number of composited samples (so the termination
                                       stops) -- equal for two inputs only if, almost surely,
                                       no piece boundary lies between them */
} orc_args;

/* ------------------------------------------------------------------------------------------ */
/* FP32 decision arithmetic.  volatile temporaries keep every operation a separately rounded   */
/* IEEE binary32 operation (the library is also built with -ffp-contract=off).                */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    float R[3][3], t[3];
    int proj, W, H;
    float half_w, half_h;   /* ortho */
    float th_w, th;         /* persp: tan(fov/2) * aspect, tan(fov/2) */
} cam32;

static float f_add(float a, float b) { volatile float r = a + b; return r; }
static float f_sub(float a, float b) { volatile float r = a - b; return r; }
static float f_mul(float a, float b) { volatile float r = a * b; return r; }
static float f_div(float a, float b) { volatile float r = a / b; return r; }

static void cam_setup(cam32 *c, const orc_args *a) {
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c->R[r][k] = a->view[r * 4 + k];
        c->t[r] = a->view[r * 4 + 3];
    }
    c->proj = a->proj; c->W = a->W; c->H = a->H;
    float aspect = f_div((float)a->W, (float)a->H);
    c->half_h = f_mul(a->param, 0.5f);
    c->half_w = f_mul(c->half_h, aspect);
    /* tan is evaluated once on the host in double and rounded to float */
    c->th = (float)tan((double)a->param * 0.5);
    c->th_w = f_mul(c->th, aspect);
}

/* Pixel (i, j): column i, row j (row 0 at the top).  Image-plane point through the pixel
 * centre; orthographic rays are parallel to the view axis, perspective rays leave the eye. */
static void ray32(const cam32 *c, int64_t i, int64_t j, float o[3], float d[3]) {
    float sx = f_sub(f_mul(f_div(f_add((float)i, 0.5f), (float)c->W), 2.0f), 1.0f);
    float sy = f_sub(1.0f, f_mul(f_div(f_add((float)j, 0.5f), (float)c->H), 2.0f));
    float e[3], de[3];
    if (c->proj == 0) {
        e[0] = f_mul(sx, c->half_w); e[1] = f_mul(sy, c->half_h); e[2] = 0.0f;
        de[0] = 0.0f; de[1] = 0.0f; de[2] = -1.0f;
    } else {
        e[0] = e[1] = e[2] = 0.0f;
        float x = f_mul(sx, c->th_w), y = f_mul(sy, c->th), z = -1.0f;
        float n2 = f_add(f_add(f_mul(x, x), f_mul(y, y)), f_mul(z, z));
        volatile float len = sqrtf(n2);
        de[0] = f_div(x, len); de[1] = f_div(y, len); de[2] = f_div(z, len);
    }
    float y0 = f_sub(e[0], c->t[0]), y1 = f_sub(e[1], c->t[1]), y2 = f_sub(e[2], c->t[2]);
    for (int k = 0; k < 3; ++k) {
        /* world = R^T (eye - t) */
        o[k] = f_add(f_add(f_mul(c->R[0][k], y0), f_mul(c->R[1][k], y1)), f_mul(c->R[2][k], y2));
        d[k] = f_add(f_add(f_mul(c->R[0][k], de[0]), f_mul(c->R[1][k], de[1])),
                     f_mul(c->R[2][k], de[2]));
    }
}

/* Slab interval of one axis for the half-open coordinate range [lo, hi).
 * Returns 0 if the ray can never be inside (parallel and outside). */
static int slab32(float o, float d, float lo, float hi, float *entry, float *exit_) {
    if (d == 0.0f) {
        if (lo <= o && o < hi) { *entry = -INFINITY; *exit_ = INFINITY; return 1; }
        return 0;
    }
    float t0 = f_div(f_sub(lo, o), d), t1 = f_div(f_sub(hi, o), d);
    *entry = t0 < t1 ? t0 : t1;
    *exit_ = t0 < t1 ? t1 : t0;
    return 1;
}

static int64_t kceil(float t, float step) {
    float q = ceilf(f_div(t, step));
    if (q > 4.0e18f) return (int64_t)4000000000000000000LL;   /* only for near-parallel axes */
    if (q < -4.0e18f) return -(int64_t)4000000000000000000LL;
    return (int64_t)q;
}

/* Lattice range [k0, k1) of samples inside the box [lo, hi) (t >= 0).  Returns 0 if empty. */
static int box_krange(const float o[3], const float d[3], const float lo[3], const float hi[3],
                      float step, int64_t *k0, int64_t *k1) {
    float tin = 0.0f, tout = INFINITY;
    for (int a = 0; a < 3; ++a) {
        float en, ex;
        if (!slab32(o[a], d[a], lo[a], hi[a], &en, &ex)) return 0;
        if (en > tin) tin = en;
        if (ex < tout) tout = ex;
    }
    if (!(tout > tin) || !(tout < INFINITY)) return 0;   /* zero direction: no samples */
    *k0 = kceil(tin, step);
    *k1 = kceil(tout, step);
    return *k1 > *k0;
}

/* ------------------------------------------------------------------------------------------ */
/* Rounding to binary16 / bfloat16, nearest-even, from the formats' definitions.              */
/* ------------------------------------------------------------------------------------------ */
static float round_to_format(float x, int mant_bits, int emin, float ovf) {
    if (!isfinite(x) || x == 0.0f) return x;
    float ax = fabsf(x);
    int e;
    frexpf(ax, &e);                         /* ax = m 2^e, m in [0.5, 1) */
    int qe = (e - 1) - mant_bits;           /* spacing of representable values near ax */
    int qmin = emin - mant_bits;            /* spacing of the subnormals */
    if (qe < qmin) qe = qmin;
    float q = ldexpf(1.0f, qe);
    float r = rintf(ax / q) * q;            /* ax/q exact; rintf rounds half to even */
    if (ax >= ovf) r = INFINITY;            /* at or above max + half a spacing */
    return x < 0 ? -r : r;
}
float orc_round_fp16(float x) { return round_to_format(x, 10, -14, 65520.0f); }
/* bfloat16: rounding up past the largest finite value overflows the float product to inf */
float orc_round_bf16(float x) { return round_to_format(x, 7, -126, INFINITY); }

/* Power-of-two scale exponent of a brick: FP16 maps max|v| to at most 2^14, BF16 to at most 1.
 * ceil(log2 m) from the exact frexp decomposition. */
int orc_scale_exponent(float maxabs, int quant) {
    if (!(maxabs > 0.0f)) return 0;
    int e;
    float m = frexpf(maxabs, &e);
    int cl = (m == 0.5f) ? e - 1 : e;       /* ceil(log2 maxabs) */
    return quant == 1 ? cl - 14 : cl;
}

/* Per-brick exponents for a brick grid of core size b with ghost g (stored region clamped to
 * the cube).  exps has nbx*nby*nbz entries, brick index = cx + nbx*(cy + nby*cz). */
void orc_brick_exponents(const float *vox, int64_t nx, int64_t ny, int64_t nz, int64_t bx,
                         int64_t by, int64_t bz, int ghost, int quant, int32_t *exps) {
    int64_t nbx = (nx + bx - 1) / bx, nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
    for (int64_t cz = 0; cz < nbz; ++cz)
        for (int64_t cy = 0; cy < nby; ++cy)
            for (int64_t cx = 0; cx < nbx; ++cx) {
                int64_t x0 = cx * bx - ghost, x1 = (cx + 1) * bx + ghost;
                int64_t y0 = cy * by - ghost, y1 = (cy + 1) * by + ghost;
                int64_t z0 = cz * bz - ghost, z1 = (cz + 1) * bz + ghost;
                x0 = x0 < 0 ? 0 : x0; y0 = y0 < 0 ? 0 : y0; z0 = z0 < 0 ? 0 : z0;
                x1 = x1 > nx ? nx : x1; y1 = y1 > ny ? ny : y1; z1 = z1 > nz ? nz : z1;
                float m = 0.0f;
                for (int64_t z = z0; z < z1; ++z)
                    for (int64_t y = y0; y < y1; ++y)
                        for (int64_t x = x0; x < x1; ++x) {
                            float v = fabsf(vox[x + nx * (y + ny * z)]);
                            if (v > m) m = v;
                        }
                exps[cx + nbx * (cy + nby * cz)] = orc_scale_exponent(m, quant);
            }
}

/* Stored code of voxel value v in a brick with exponent e, as a float. */
static float quant_code(float v, int e, int quant) {
    float s = ldexpf(v, -e);                /* exact power-of-two scaling */
    return quant == 1 ? orc_round_fp16(s) : orc_round_bf16(s);
}

void orc_minmax(const float *v, int64_t n, float *vmin, float *vmax) {
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if (v[i] < lo) lo = v[i];
        if (v[i] > hi) hi = v[i];
    }
    *vmin = lo; *vmax = hi;
}

/* ------------------------------------------------------------------------------------------ */
/* Sample enumeration                                                                         */
/* ------------------------------------------------------------------------------------------ */
#define MAXCELLS 4096
typedef struct {
    float o[3], d[3];
    int64_t k0, k1;                 /* samples in the cube */
    int64_t nb[3];
    int64_t b[3];                   /* brick core size per axis (n if unbricked) */
    /* per axis, per cell: lattice range [ke, kx) owned by that cell */
    int64_t *ke[3], *kx[3];
    int inside0[3];                 /* d == 0: index of the cell holding o, else -1 */
} rayinfo;

/* Window of the render along axis ax: [wlo, whi) clipped to the cube (the whole axis if no
 * window is set).  Section 2.3: the user views the whole cube or a sub-cube. */
static void window_axis(const orc_args *a, int ax, int64_t n, int64_t *wlo, int64_t *whi) {
    int has = a->win_hi[0] > a->win_lo[0] && a->win_hi[1] > a->win_lo[1] && a->win_hi[2] > a->win_lo[2];
    *wlo = has ? (a->win_lo[ax] > 0 ? a->win_lo[ax] : 0) : 0;
    *whi = has ? (a->win_hi[ax] < n ? a->win_hi[ax] : n) : n;
}

static int ray_setup(const orc_args *a, const cam32 *c, int64_t pix, rayinfo *r,
                     int64_t *buf) {
    int64_t i = pix % a->W, j = pix / a->W;
    ray32(c, i, j, r->o, r->d);
    int64_t n[3] = {a->nx, a->ny, a->nz};
    int64_t bb[3] = {a->bx, a->by, a->bz};
    int64_t wl[3], wh[3];
    for (int ax = 0; ax < 3; ++ax) window_axis(a, ax, n[ax], &wl[ax], &wh[ax]);
    float lo[3] = {(float)wl[0], (float)wl[1], (float)wl[2]};
    float hi[3] = {(float)wh[0], (float)wh[1], (float)wh[2]};
    if (!(wh[0] > wl[0] && wh[1] > wl[1] && wh[2] > wl[2])) { r->k0 = r->k1 = 0; }
    else if (!box_krange(r->o, r->d, lo, hi, a->step, &r->k0, &r->k1)) { r->k0 = r->k1 = 0; }
    int64_t off = 0;
    for (int ax = 0; ax < 3; ++ax) {
        r->b[ax] = bb[ax] > 0 ? bb[ax] : n[ax];
        r->nb[ax] = (n[ax] + r->b[ax] - 1) / r->b[ax];
        r->ke[ax] = buf + off; off += r->nb[ax];
        r->kx[ax] = buf + off; off += r->nb[ax];
        r->inside0[ax] = -1;
        for (int64_t cc = 0; cc < r->nb[ax]; ++cc) {
            /* the cell's planes, clipped to the window (shared planes stay identical) */
            int64_t l = cc * r->b[ax], h = (cc + 1) * r->b[ax];
            if (h > n[ax]) h = n[ax];
            if (l < wl[ax]) l = wl[ax];
            if (h > wh[ax]) h = wh[ax];
            float plo = (float)l, phi = (float)h;
            float en, ex;
            if (h <= l || !slab32(r->o[ax], r->d[ax], plo, phi, &en, &ex)) {
                r->ke[ax][cc] = 1; r->kx[ax][cc] = 0;  /* empty */
                continue;
            }
            if (r->d[ax] == 0.0f) {
                r->inside0[ax] = (int)cc;
                r->ke[ax][cc] = INT64_MIN; r->kx[ax][cc] = INT64_MAX;
            } else {
                r->ke[ax][cc] = kceil(en, a->step);
                r->kx[ax][cc] = kceil(ex, a->step);
            }
        }
    }
    return r->k1 > r->k0;
}

/* Cell along one axis owning lattice index k (exactly one must match). */
static int64_t owner_cell(const rayinfo *r, int ax, int64_t k) {
    int64_t found = -1;
    for (int64_t cc = 0; cc < r->nb[ax]; ++cc)
        if (r->ke[ax][cc] <= k && k < r->kx[ax][cc]) {
            if (found >= 0) return -2;     /* overlap: the partition is broken */
            found = cc;
        }
    return found;
}

/* ------------------------------------------------------------------------------------------ */
/* Procedural cube (the out-of-core stand-in for cubes larger than HBM).  An input generator,   */
/* not part of the method: defined here from its published parts, independently of the        */
/* renderer's own copy.                                                                         */
/*   SplitMix64 (Steele, Lea & Flood 2014): state += 0x9E3779B97F4A7C15, then the two          */
/*   xor-shift-multiply rounds and a final xor-shift.                                           */
/*   noise(x,y,z): c = (z*ny + y)*ceil(nx/2) + floor(x/2); h = SplitMix64 of the state         */
/*   c ^ (seed * 0xD1B54A32D192ED03); u1 = (h>>40 + 1/2) 2^-24, u2 = ((h>>16) & 0xFFFFFF) 2^-24; */
/*   Box-Muller: r = sqrt(-2 ln u1), even x -> r cos(2 pi u2), odd x -> r sin(2 pi u2).        */
/*   sources: 4 per 256^3 cell q = (qz*ncy + qy)*ncx + qx, drawn from the SplitMix64 stream   */
/*   seeded with seed ^ (q * 0x9E3779B97F4A7C15) ^ 0x632BE59BD9B4E019, six uniforms each       */
/*   (top 53 bits): centre (q + u) 256, sigma_xy = 1 + 3u, sigma_z = sigma_xy (2 + 3u),        */
/*   amplitude exp(ln 3 + (ln 100 - ln 3) u); a source adds amp exp(-r^2/2) to voxels with    */
/*   |dx|,|dy| <= 4 sigma_xy and |dz| <= 4 sigma_z (d from the voxel centre).                  */
/*   voxel = (float)(noise + the sources in increasing (q, k) order).                          */
/* ------------------------------------------------------------------------------------------ */
static uint64_t sm64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define PROC_CELL 256
#define PROC_K 4
typedef struct { double cx, cy, cz, sxy, sz, amp; } psrc;

static void proc_cell_sources(uint64_t seed, int64_t qx, int64_t qy, int64_t qz, int64_t ncx,
                              int64_t ncy, psrc out[PROC_K]) {
    uint64_t q = (uint64_t)((qz * ncy + qy) * ncx + qx);
    uint64_t st = seed ^ (q * 0x9E3779B97F4A7C15ULL) ^ 0x632BE59BD9B4E019ULL;
    for (int k = 0; k < PROC_K; ++k) {
        double u[6];
        for (int i = 0; i < 6; ++i) u[i] = (double)(sm64_next(&st) >> 11) * 0x1.0p-53;
        out[k].cx = ((double)qx + u[0]) * PROC_CELL;
        out[k].cy = ((double)qy + u[1]) * PROC_CELL;
        out[k].cz = ((double)qz + u[2]) * PROC_CELL;
        out[k].sxy = 1.0 + 3.0 * u[3];
        out[k].sz = out[k].sxy * (2.0 + 3.0 * u[4]);
        out[k].amp = exp(log(3.0) + (log(100.0) - log(3.0)) * u[5]);
    }
}

static double proc_noise(uint64_t seed, int64_t nx, int64_t ny, int64_t x, int64_t y, int64_t z) {
    uint64_t c = (uint64_t)((z * ny + y) * ((nx + 1) / 2) + (x >> 1));
    uint64_t st = c ^ (seed * 0xD1B54A32D192ED03ULL);
    uint64_t h = sm64_next(&st);
    double u1 = ((double)(h >> 40) + 0.5) * 0x1.0p-24;   /* in (0, 1): r > 0, never -0 */
    double u2 = (double)((h >> 16) & 0xFFFFFFULL) * 0x1.0p-24;
    double r = sqrt(-2.0 * log(u1));
    double th = 6.283185307179586 * u2;
    return (x & 1) ? r * sin(th) : r * cos(th);
}

static double proc_source_term(const psrc *s, int64_t x, int64_t y, int64_t z) {
    double dx = ((double)x + 0.5) - s->cx, dy = ((double)y + 0.5) - s->cy, dz = ((double)z + 0.5) - s->cz;
    if (!(fabs(dx) <= 4.0 * s->sxy && fabs(dy) <= 4.0 * s->sxy && fabs(dz) <= 4.0 * s->sz)) return 0.0;
    return s->amp * exp(-0.5 * (dx * dx / (s->sxy * s->sxy) + dy * dy / (s->sxy * s->sxy) +
                                dz * dz / (s->sz * s->sz)));
}

/* One voxel of the procedural cube (the sources of the 27 cells around the voxel's cell, in
 * increasing cell order; farther cells cannot reach it: 4 sigma <= 80 < 256). */
float orc_proc_voxel(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y,
                     int64_t z) {
    /* per-thread copy of the last neighbourhood's sources (cells in increasing order) */
    static __thread uint64_t c_seed;
    static __thread int64_t c_key[6] = {-1, -1, -1, -1, -1, -1};
    static __thread psrc c_src[27 * PROC_K];
    static __thread int c_n;
    int64_t ncx = (nx + PROC_CELL - 1) / PROC_CELL, ncy = (ny + PROC_CELL - 1) / PROC_CELL,
            ncz = (nz + PROC_CELL - 1) / PROC_CELL;
    int64_t qx = x / PROC_CELL, qy = y / PROC_CELL, qz = z / PROC_CELL;
    if (c_seed != seed || c_key[0] != qx || c_key[1] != qy || c_key[2] != qz || c_key[3] != nx ||
        c_key[4] != ny || c_key[5] != nz) {
        c_n = 0;
        for (int64_t cz = qz - 1; cz <= qz + 1; ++cz)
            for (int64_t cy = qy - 1; cy <= qy + 1; ++cy)
                for (int64_t cx = qx - 1; cx <= qx + 1; ++cx) {
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= ncx || cy >= ncy || cz >= ncz) continue;
                    proc_cell_sources(seed, cx, cy, cz, ncx, ncy, &c_src[c_n]);
                    c_n += PROC_K;
                }
        c_seed = seed;
        c_key[0] = qx; c_key[1] = qy; c_key[2] = qz; c_key[3] = nx; c_key[4] = ny; c_key[5] = nz;
    }
    double v = proc_noise(seed, nx, ny, x, y, z);
    for (int i = 0; i < c_n; ++i) v += proc_source_term(&c_src[i], x, y, z);
    return (float)v;
}

double orc_proc_noise(uint64_t seed, int64_t nx, int64_t ny, int64_t x, int64_t y, int64_t z) {
    return proc_noise(seed, nx, ny, x, y, z);
}

/* The voxels of the box [lo, lo + dim) with coordinates clamped to the cube, x fastest. */
void orc_proc_region(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, const int64_t lo[3],
                     const int64_t dim[3], float *out) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < dim[1] * dim[2]; ++r) {
        int64_t y = lo[1] + r % dim[1], z = lo[2] + r / dim[1];
        y = y < 0 ? 0 : (y >= ny ? ny - 1 : y);
        z = z < 0 ? 0 : (z >= nz ? nz - 1 : z);
        for (int64_t i = 0; i < dim[0]; ++i) {
            int64_t x = lo[0] + i;
            x = x < 0 ? 0 : (x >= nx ? nx - 1 : x);
            out[r * dim[0] + i] = orc_proc_voxel(seed, nx, ny, nz, x, y, z);
        }
    }
}

/* Voxel value at flat index idx of the cube described by a (array or procedural). */
static float vox_at(const orc_args *a, int64_t idx) {
    if (!a->procedural) return a->vox[idx];
    int64_t x = idx % a->nx, y = (idx / a->nx) % a->ny, z = idx / (a->nx * a->ny);
    return orc_proc_voxel(a->proc_seed, a->nx, a->ny, a->nz, x, y, z);
}

/* ------------------------------------------------------------------------------------------ */
/* Field evaluation                                                                           */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t idx[8];                 /* flat voxel index of the 8 corners (after clamping) */
    double w[8];                    /* trilinear weights */
    double v;                       /* interpolated value */
} tri64;

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* A disabled spectral channel (Section 2.3: channels switched off like a colour-map change)
 * holds vmin, the bottom of the table range, in place of its data. */
static int channel_off(const orc_args *a, int64_t idx) {
    return a->channels && !a->channels[idx / (a->nx * a->ny)];
}

/* voxel value as seen from a brick (dequantised with the brick's exponent when quantised) */
static double voxel_val(const orc_args *a, int64_t idx, int e) {
    if (channel_off(a, idx)) return (double)a->vmin;
    float v = vox_at(a, idx);
    if (a->quant == 0) return (double)v;
    return ldexp((double)quant_code(v, e, a->quant), e);
}

static void trilinear64(const orc_args *a, const double p[3], int e, tri64 *t) {
    int64_t n[3] = {a->nx, a->ny, a->nz};
    int64_t i0[3], i1[3];
    double f[3];
    for (int ax = 0; ax < 3; ++ax) {
        double x = p[ax] - 0.5;
        double fl = floor(x);
        f[ax] = x - fl;
        i0[ax] = clampi((int64_t)fl, 0, n[ax] - 1);
        i1[ax] = clampi((int64_t)fl + 1, 0, n[ax] - 1);
    }
    double v = 0.0;
    for (int c = 0; c < 8; ++c) {
        int64_t xi = (c & 1) ? i1[0] : i0[0];
        int64_t yi = (c & 2) ? i1[1] : i0[1];
        int64_t zi = (c & 4) ? i1[2] : i0[2];
        double w = ((c & 1) ? f[0] : 1.0 - f[0]) * ((c & 2) ? f[1] : 1.0 - f[1]) *
                   ((c & 4) ? f[2] : 1.0 - f[2]);
        int64_t idx = xi + n[0] * (yi + n[1] * zi);
        t->idx[c] = idx;
        t->w[c] = w;
        v += w * voxel_val(a, idx, e);
    }
    t->v = v;
}

/* The FP32 operation order used by MIP: global position o + fl(k*step)*d, then linear
 * interpolation a + f*(b-a) along x, then y, then z, every step rounded to binary32. */
static float lerp32(float a, float b, float f) { return f_add(a, f_mul(f, f_sub(b, a))); }

static float sample32(const orc_args *a, const float o[3], const float d[3], int64_t k, int e) {
    int64_t n[3] = {a->nx, a->ny, a->nz};
    float t = f_mul((float)k, a->step);
    int64_t i0[3], i1[3];
    float f[3];
    for (int ax = 0; ax < 3; ++ax) {
        float p = f_add(o[ax], f_mul(t, d[ax]));
        float x = f_sub(p, 0.5f);
        float fl = floorf(x);
        f[ax] = f_sub(x, fl);
        i0[ax] = clampi((int64_t)fl, 0, n[ax] - 1);
        i1[ax] = clampi((int64_t)fl + 1, 0, n[ax] - 1);
    }
    float c[8];
    for (int cc = 0; cc < 8; ++cc) {
        int64_t idx = ((cc & 1) ? i1[0] : i0[0]) +
                      n[0] * (((cc & 2) ? i1[1] : i0[1]) + n[1] * ((cc & 4) ? i1[2] : i0[2]));
        float v = vox_at(a, idx);
        c[cc] = a->quant ? quant_code(v, e, a->quant) : v;
        if (channel_off(a, idx)) c[cc] = a->quant ? ldexpf(a->vmin, -e) : a->vmin;
    }
    float c00 = lerp32(c[0], c[1], f[0]), c10 = lerp32(c[2], c[3], f[0]);
    float c01 = lerp32(c[4], c[5], f[0]), c11 = lerp32(c[6], c[7], f[0]);
    float c0 = lerp32(c00, c10, f[1]), c1 = lerp32(c01, c11, f[1]);
    float v = lerp32(c0, c1, f[2]);
    return a->quant ? ldexpf(v, e) : v;
}

/* Transfer function: u = clamp((v - vmin)/(vmax - vmin)), x = u (N-1), linear between the two
 * neighbouring entries. */
typedef struct { double rgba[4]; int64_t i; double f; double dxdv; } tf64;

static void tf_eval(const orc_args *a, double v, tf64 *r) {
    double range = (double)a->vmax - (double)a->vmin;
    double u = (v - (double)a->vmin) / range;
    double dudv = 1.0 / range;
    if (u <= 0.0) { u = 0.0; dudv = 0.0; }
    if (u >= 1.0) { u = 1.0; dudv = 0.0; }
    double x = u * (double)(a->nlut - 1);
    int64_t i = (int64_t)floor(x);
    if (i > a->nlut - 2) i = a->nlut - 2;
    double f = x - (double)i;
    for (int ch = 0; ch < 4; ++ch)
        r->rgba[ch] = (1.0 - f) * (double)a->lut[i * 4 + ch] + f * (double)a->lut[(i + 1) * 4 + ch];
    r->i = i; r->f = f; r->dxdv = dudv * (double)(a->nlut - 1);
}

/* ------------------------------------------------------------------------------------------ */
/* One pixel                                                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    tri64 tri; tf64 tf; double Tb;  /* transmittance before this sample */
} smp;

enum { FLAG_ERT_FRAGILE = 1, FLAG_NO_SAMPLES = 2, FLAG_PARTITION_ERROR = 4, FLAG_TABLE_KINK = 8 };

/* Half-width, in table-coordinate units, of the band around a table entry inside which the
 * interval a sample falls in may differ between this FP64 trilinear value and a binary32 one
 * (whose error is ~1e-6 of the value range here): the image is continuous there, its
 * derivative with respect to the value is not. */
#define TABLE_KINK_BAND 1e-4

/* Traces one pixel.  If keep != NULL, the composited samples are stored there (capacity cap). */
static int pixel_trace(const orc_args *a, const cam32 *c, const int32_t *exps, int64_t pix,
                       int64_t *buf, double out[4], uint8_t *flag, int64_t *ns,
                       smp *keep, int64_t cap, int64_t *nkeep, uint64_t *sig) {
    uint64_t h = 0xCBF29CE484222325ULL;     /* FNV-1a over the pieces of the composited samples */
    rayinfo r;
    *flag = 0; *ns = 0;
    if (nkeep) *nkeep = 0;
    int hit = ray_setup(a, c, pix, &r, buf);
    double thr = (double)f_sub(1.0f, a->tau < 1.0f ? a->tau : 1.0f);
    double fragile_band = 2e-4 * thr;
    if (a->mode != 0) {
        double m = -INFINITY;
        float m32 = -INFINITY;
        for (int64_t k = r.k0; hit && k < r.k1; ++k) {
            int64_t cx = owner_cell(&r, 0, k), cy = owner_cell(&r, 1, k), cz = owner_cell(&r, 2, k);
            if (cx < 0 || cy < 0 || cz < 0) { *flag |= FLAG_PARTITION_ERROR; continue; }
            int e = exps ? exps[cx + r.nb[0] * (cy + r.nb[1] * cz)] : 0;
            if (a->mode == 2) {
                float v = sample32(a, r.o, r.d, k, e);
                if (v > m32) m32 = v;
            } else {
                double p[3];
                for (int ax = 0; ax < 3; ++ax)
                    p[ax] = (double)r.o[ax] + ((double)k * (double)a->step) * (double)r.d[ax];
                tri64 t;
                trilinear64(a, p, e, &t);
                if (t.v > m) m = t.v;
            }
            ++*ns;
        }
        if (a->mode == 2) m = (double)m32;
        if (*ns == 0) { *flag |= FLAG_NO_SAMPLES; m = (double)a->vmin; }
        out[0] = m;
        return 0;
    }
    double C[3] = {0, 0, 0}, T = 1.0;      /* global */
    double Tseg = 1.0;                      /* transmittance of the current brick segment */
    int64_t seg[3] = {-1, -1, -1};
    int stopped = 0;
    for (int64_t k = r.k0; hit && k < r.k1; ++k) {
        int64_t cx = owner_cell(&r, 0, k), cy = owner_cell(&r, 1, k), cz = owner_cell(&r, 2, k);
        if (cx < 0 || cy < 0 || cz < 0) { *flag |= FLAG_PARTITION_ERROR; continue; }
        if (cx != seg[0] || cy != seg[1] || cz != seg[2]) {  /* a new brick segment */
            seg[0] = cx; seg[1] = cy; seg[2] = cz;
            /* per-segment termination restarts from full transmittance in every brick (the
             * parts are ray-cast independently, Section 2.5); global termination keeps the
             * whole ray's transmittance and its stop (Section 2.4) */
            if (!a->term_global) { Tseg = 1.0; stopped = 0; }
        }
        if (stopped) continue;
        int e = exps ? exps[cx + r.nb[0] * (cy + r.nb[1] * cz)] : 0;
        double p[3];
        for (int ax = 0; ax < 3; ++ax)
            p[ax] = (double)r.o[ax] + ((double)k * (double)a->step) * (double)r.d[ax];
        smp s;
        trilinear64(a, p, e, &s.tri);
        tf_eval(a, s.tri.v, &s.tf);
        double al = s.tf.rgba[3];
        s.Tb = T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * al * s.tf.rgba[ch];
        T *= (1.0 - al);
        Tseg *= (1.0 - al);
        ++*ns;
        if (keep && *nkeep < cap) keep[(*nkeep)++] = s;
        if (sig) {
            double u = (s.tri.v - (double)a->vmin) / ((double)a->vmax - (double)a->vmin);
            uint64_t piece = u <= 0.0 ? 0 : (u >= 1.0 ? (uint64_t)a->nlut : (uint64_t)s.tf.i + 1);
            h = (h ^ piece) * 0x100000001B3ULL;
        }
        {
            double xr = (s.tri.v - (double)a->vmin) / ((double)a->vmax - (double)a->vmin) * (double)(a->nlut - 1);
            if (xr > -0.5 && xr < (double)a->nlut - 0.5 && fabs(xr - nearbyint(xr)) < TABLE_KINK_BAND)
                *flag |= FLAG_TABLE_KINK;
        }
        if (thr > 0.0 && fabs(Tseg - thr) <= fragile_band) *flag |= FLAG_ERT_FRAGILE;
        if (Tseg <= thr) stopped = 1;
    }
    if (*ns == 0) *flag |= FLAG_NO_SAMPLES;
    if (sig) *sig = (h ^ (uint64_t)*ns) * 0x100000001B3ULL;
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    return 0;
}

static int64_t bufsize(const orc_args *a) {
    int64_t n[3] = {a->nx, a->ny, a->nz}, b[3] = {a->bx, a->by, a->bz}, s = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int64_t bb = b[ax] > 0 ? b[ax] : n[ax];
        s += 2 * ((n[ax] + bb - 1) / bb);
    }
    return s;
}

static int32_t *make_exps(const orc_args *a) {
    if (a->quant == 0 || a->procedural) return NULL;
    int64_t bx = a->bx > 0 ? a->bx : a->nx, by = a->by > 0 ? a->by : a->ny,
            bz = a->bz > 0 ? a->bz : a->nz;
    int64_t nb = ((a->nx + bx - 1) / bx) * ((a->ny + by - 1) / by) * ((a->nz + bz - 1) / bz);
    int32_t *e = (int32_t *)malloc(sizeof(int32_t) * nb);
    orc_brick_exponents(a->vox, a->nx, a->ny, a->nz, bx, by, bz, a->ghost, a->quant, e);
    return e;
}

/* Renders the listed pixels (pix = row*W + col; NULL = every pixel in order).
 * out: npix x 4 (DVR: premultiplied r, g, b, alpha) or npix x 1 (MIP).
 * flags: per pixel, bit0 = ERT decision within 2e-4 (relative) of the threshold,
 * bit1 = no samples, bit2 = broken sample partition (never expected), bit3 = a composited DVR
 * sample's table coordinate within TABLE_KINK_BAND of an entry (its gradient is ambiguous). */
int orc_render(const orc_args *a, const int64_t *pix, int64_t npix, double *out, uint8_t *flags,
               int64_t *nsamples) {
    if (a->nlut < 2 || a->W <= 0 || a->H <= 0 || !(a->step > 0.0f)) return -1;
    if (a->procedural && a->quant) return -2;
    cam32 c;
    cam_setup(&c, a);
    int32_t *exps = make_exps(a);
    int64_t bs = bufsize(a);
    int stride = a->mode == 0 ? 4 : 1;
    int64_t total = 0;
#ifdef _OPENMP
    int nt = a->nthreads > 0 ? a->nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt) reduction(+ : total)
#endif
    {
        int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * bs);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t q = 0; q < npix; ++q) {
            int64_t p = pix ? pix[q] : q;
            int64_t ns;
            pixel_trace(a, &c, exps, p, buf, out + q * stride, flags + q, &ns, NULL, 0, NULL,
                        a->sig ? a->sig + q : NULL);
            total += ns;
        }
        free(buf);
    }
    if (nsamples) *nsamples = total;
    free(exps);
    return 0;
}

/* Reverse-mode gradient of sum_p <gout[p], out[p]> (DVR, FP32 voxels) with respect to the table
 * (glut, nlut x 4) and the voxels (gvox, nx*ny*nz, may be NULL).  The early-termination stop of
 * every segment is held fixed (the output is piecewise smooth in the inputs). */
int orc_render_grad(const orc_args *a, const int64_t *pix, int64_t npix, const double *gout,
                    double *glut, double *gvox) {
    if (a->mode != 0 || a->quant != 0) return -1;
    cam32 c;
    cam_setup(&c, a);
    int64_t bs = bufsize(a);
    int64_t nvox = a->nx * a->ny * a->nz;
    int64_t cap = 4 * (a->nx + a->ny + a->nz) * (int64_t)(2.0f / a->step + 2.0f) + 64;
    memset(glut, 0, sizeof(double) * 4 * a->nlut);
    if (gvox) memset(gvox, 0, sizeof(double) * nvox);
    /* serial over pixels: the voxel gradient is a scatter */
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * bs);
    smp *keep = (smp *)malloc(sizeof(smp) * cap);
    for (int64_t q = 0; q < npix; ++q) {
        int64_t p = pix ? pix[q] : q;
        double out[4];
        uint8_t flag;
        int64_t ns, nk;
        pixel_trace(a, &c, NULL, p, buf, out, &flag, &ns, keep, cap, &nk, NULL);
        const double *g = gout + 4 * q;
        double T_final = 1.0 - out[3];
        double gT = -g[3];                  /* A = 1 - T_final */
        (void)T_final;
        for (int64_t m = nk - 1; m >= 0; --m) {
            const smp *s = &keep[m];
            double al = s->tf.rgba[3], Tb = s->Tb;
            double gc_dot = g[0] * s->tf.rgba[0] + g[1] * s->tf.rgba[1] + g[2] * s->tf.rgba[2];
            double grgba[4];
            for (int ch = 0; ch < 3; ++ch) grgba[ch] = g[ch] * Tb * al;
            grgba[3] = Tb * gc_dot - gT * Tb;
            gT = gT * (1.0 - al) + al * gc_dot;
            int64_t i = s->tf.i;
            double f = s->tf.f, dvdx = 0.0;
            for (int ch = 0; ch < 4; ++ch) {
                glut[i * 4 + ch] += (1.0 - f) * grgba[ch];
                glut[(i + 1) * 4 + ch] += f * grgba[ch];
                dvdx += grgba[ch] * ((double)a->lut[(i + 1) * 4 + ch] - (double)a->lut[i * 4 + ch]);
            }
            if (gvox) {
                double gv = dvdx * s->tf.dxdv;
                for (int cc = 0; cc < 8; ++cc)
                    if (!channel_off(a, s->tri.idx[cc])) gvox[s->tri.idx[cc]] += s->tri.w[cc] * gv;
            }
        }
    }
    free(keep);
    free(buf);
    return 0;
}

/* Rays of the listed pixels in the FP32 decision arithmetic (o, d: npix x 3) and their lattice
 * range inside the cube (k: npix x 2; k0 == k1 when the ray misses). */
void orc_rays(const orc_args *a, const int64_t *pix, int64_t npix, float *o, float *d,
              int64_t *k) {
    cam32 c;
    cam_setup(&c, a);
    float lo[3] = {0, 0, 0}, hi[3] = {(float)a->nx, (float)a->ny, (float)a->nz};
    for (int64_t q = 0; q < npix; ++q) {
        int64_t p = pix ? pix[q] : q;
        ray32(&c, p % a->W, p / a->W, o + 3 * q, d + 3 * q);
        int64_t k0 = 0, k1 = 0;
        if (!box_krange(o + 3 * q, d + 3 * q, lo, hi, a->step, &k0, &k1)) k0 = k1 = 0;
        k[2 * q] = k0; k[2 * q + 1] = k1;
    }
}

/* Owning brick (cx, cy, cz) of every sample of one pixel, in lattice order (owners: n x 3). */
int64_t orc_sample_owners(const orc_args *a, int64_t pix, int64_t *owners, int64_t cap) {
    cam32 c;
    cam_setup(&c, a);
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * bufsize(a));
    rayinfo r;
    int64_t n = 0;
    if (ray_setup(a, &c, pix, &r, buf))
        for (int64_t k = r.k0; k < r.k1 && n < cap; ++k, ++n)
            for (int ax = 0; ax < 3; ++ax) owners[3 * n + ax] = owner_cell(&r, ax, k);
    free(buf);
    return n;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Lossy wavelet block store (Section 6: wavelet compression of the cube portions kept in GPU   */
/* memory, decompressible with random access).  The format is the one the library documents:  */
/* 8x8x8 blocks on a global grid (upper-face blocks repeat the edge voxels), three levels of    */
/* the 3D Haar average/difference transform in binary32, int8 detail codes with one            */
/* power-of-two step per subband, the block average in FP32, one 544-byte record per block.    */
/* Written from that definition; every binary32 operation is a separate rounded step.          */
/* ------------------------------------------------------------------------------------------ */
#define WREC 544

static float f_half(float v) { volatile float r = v * 0.5f; return r; }

/* One line of n values at stride st: forward pairs (2i, 2i+1) -> (i, n/2 + i). */
static void haar_line_fwd(float *w, int base, int st, int n) {
    float tmp[8];
    int h = n / 2;
    for (int i = 0; i < h; ++i) {
        float a = w[base + (2 * i) * st], b = w[base + (2 * i + 1) * st];
        tmp[i] = f_half(f_add(a, b));
        tmp[h + i] = f_half(f_sub(a, b));
    }
    for (int i = 0; i < n; ++i) w[base + i * st] = tmp[i];
}

/* One line, inverse: (i, n/2 + i) = (s, d) -> (2i, 2i+1) = (s + d, s - d). */
static void haar_line_inv(float *w, int base, int st, int n) {
    float tmp[8];
    int h = n / 2;
    for (int i = 0; i < h; ++i) {
        float s = w[base + i * st], d = w[base + (h + i) * st];
        tmp[2 * i] = f_add(s, d);
        tmp[2 * i + 1] = f_sub(s, d);
    }
    for (int i = 0; i < n; ++i) w[base + i * st] = tmp[i];
}

/* Pyramid index x + 8y + 64z: -1 for the average, else 7 (level - 1) + (bx + 2by + 4bz) - 1. */
static int w_subband(int x, int y, int z) {
    for (int L = 1; L <= 3; ++L) {
        int n = 8 >> (L - 1), h = n / 2;
        if (x < n && y < n && z < n && (x >= h || y >= h || z >= h))
            return 7 * (L - 1) + ((x >= h) + 2 * (y >= h) + 4 * (z >= h)) - 1;
    }
    return -1;
}

int64_t orc_wavelet_bytes(int64_t nx, int64_t ny, int64_t nz) {
    return ((nx + 7) / 8) * ((ny + 7) / 8) * ((nz + 7) / 8) * (int64_t)WREC;
}

int orc_wavelet_encode(const float *vox, int64_t nx, int64_t ny, int64_t nz, uint8_t *store) {
    int64_t bnx = (nx + 7) / 8, bny = (ny + 7) / 8, bnz = (nz + 7) / 8;
    int64_t nb = bnx * bny * bnz;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t blk = 0; blk < nb; ++blk) {
        int64_t bx = blk % bnx, by = (blk / bnx) % bny, bz = blk / (bnx * bny);
        float w[512];
        for (int z = 0; z < 8; ++z)
            for (int y = 0; y < 8; ++y)
                for (int x = 0; x < 8; ++x) {
                    int64_t gx = clampi(8 * bx + x, 0, nx - 1), gy = clampi(8 * by + y, 0, ny - 1);
                    int64_t gz = clampi(8 * bz + z, 0, nz - 1);
                    w[x + 8 * y + 64 * z] = vox[gx + nx * (gy + ny * gz)];
                }
        for (int L = 1; L <= 3; ++L) {
            int n = 8 >> (L - 1);
            for (int v = 0; v < n; ++v)            /* along x: lines over (y, z) = (u, v) */
                for (int u = 0; u < n; ++u) haar_line_fwd(w, 8 * u + 64 * v, 1, n);
            for (int v = 0; v < n; ++v)            /* along y: lines over (x, z) */
                for (int u = 0; u < n; ++u) haar_line_fwd(w, u + 64 * v, 8, n);
            for (int v = 0; v < n; ++v)            /* along z: lines over (x, y) */
                for (int u = 0; u < n; ++u) haar_line_fwd(w, u + 8 * v, 64, n);
        }
        /* per subband: the smallest e in [-126, 120] with max |c| <= 127 2^e */
        float m[21];
        for (int i = 0; i < 21; ++i) m[i] = 0.0f;
        for (int p = 1; p < 512; ++p) {
            int sb = w_subband(p & 7, (p >> 3) & 7, p >> 6);
            float a = fabsf(w[p]);
            if (a > m[sb]) m[sb] = a;
        }
        int e[21];
        for (int i = 0; i < 21; ++i) {
            if (m[i] == 0.0f) { e[i] = -128; continue; }
            int k = -126;
            while (k < 120 && m[i] > ldexpf(127.0f, k)) ++k;
            e[i] = k;
        }
        uint8_t *rec = store + blk * WREC;
        memset(rec, 0, WREC);
        for (int p = 1; p < 512; ++p) {
            int sb = w_subband(p & 7, (p >> 3) & 7, p >> 6);
            int q = 0;
            if (e[sb] != -128) {
                volatile float t = ldexpf(w[p], -e[sb]);
                q = (int)rintf(t);
                if (q > 127) q = 127;
                if (q < -127) q = -127;
            }
            rec[p] = (uint8_t)(int8_t)q;
        }
        memcpy(rec + 512, &w[0], 4);
        for (int i = 0; i < 21; ++i) rec[516 + i] = (uint8_t)(int8_t)e[i];
    }
    return 0;
}

int orc_wavelet_decode(const uint8_t *store, int64_t nx, int64_t ny, int64_t nz, float *vox) {
    int64_t bnx = (nx + 7) / 8, bny = (ny + 7) / 8, bnz = (nz + 7) / 8;
    int64_t nb = bnx * bny * bnz;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t blk = 0; blk < nb; ++blk) {
        int64_t bx = blk % bnx, by = (blk / bnx) % bny, bz = blk / (bnx * bny);
        const uint8_t *rec = store + blk * WREC;
        float w[512];
        memcpy(&w[0], rec + 512, 4);
        for (int p = 1; p < 512; ++p) {
            int sb = w_subband(p & 7, (p >> 3) & 7, p >> 6);
            int e = (int)(int8_t)rec[516 + sb];
            int q = (int)(int8_t)rec[p];
            w[p] = e == -128 ? 0.0f : ldexpf((float)q, e);
        }
        for (int L = 3; L >= 1; --L) {
            int n = 8 >> (L - 1);
            for (int v = 0; v < n; ++v)            /* along z */
                for (int u = 0; u < n; ++u) haar_line_inv(w, u + 8 * v, 64, n);
            for (int v = 0; v < n; ++v)            /* along y */
                for (int u = 0; u < n; ++u) haar_line_inv(w, u + 64 * v, 8, n);
            for (int v = 0; v < n; ++v)            /* along x */
                for (int u = 0; u < n; ++u) haar_line_inv(w, 8 * u + 64 * v, 1, n);
        }
        for (int z = 0; z < 8; ++z)
            for (int y = 0; y < 8; ++y)
                for (int x = 0; x < 8; ++x) {
                    int64_t gx = 8 * bx + x, gy = 8 * by + y, gz = 8 * bz + z;
                    if (gx < nx && gy < ny && gz < nz) vox[gx + nx * (gy + ny * gz)] = w[x + 8 * y + 64 * z];
                }
    }
    return 0;
}
