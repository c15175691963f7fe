// vr_raycast.cu -- brick ray casting (DVR and MIP) and sort-last compositing.
//
// Section 2.4: every ray inside a part's rendering rectangle is tested against the part's box;
// rays that hit are sampled between entry and exit, colours accumulated front to back, with
// early ray termination; MIP keeps the maximum sampled value.  Section 2.5: the parts'
// sub-images are blended with the associative "over" operator.
//
// Sample positions lie on the global lattice t = k*step of each ray, so which samples exist
// does not depend on the bricking.  A brick owns the lattice indices k with
// ceil(t_in/step) <= k < ceil(t_out/step), t_in/t_out from its core box's slab planes.  Those
// decisions use IEEE binary32 operations in one fixed order (the __f*_rn intrinsics are never
// contracted), identical for every brick, so neighbouring bricks split each ray's samples
// exactly, with no sample lost or counted twice.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "vr_internal.cuh"

// Tuning knobs of the ray-cast kernels (build-time): unroll factor of the DVR sample loop, the
// blocks per SM the register allocation of the fragment kernel must allow for DVR frames read
// through slice atlases and for MIP frames (0: no constraint), and the same for the one-pass
// (global termination) kernel.
#ifndef VR_SAMPLE_UNROLL
#define VR_SAMPLE_UNROLL 1
#endif
#ifndef VR_DVR_MIN_BLOCKS
#define VR_DVR_MIN_BLOCKS 6
#endif
#ifndef VR_MIP_MIN_BLOCKS
#define VR_MIP_MIN_BLOCKS 0
#endif
#ifndef VR_PAIR_PIPELINE
#define VR_PAIR_PIPELINE 1
#endif
#ifndef VR_RAYMARCH_MIN_BLOCKS
#define VR_RAYMARCH_MIN_BLOCKS 5
#endif
#ifndef VR_ADJ_MIN_BLOCKS
#define VR_ADJ_MIN_BLOCKS 4
#endif
constexpr int kSampleUnroll = VR_SAMPLE_UNROLL;

namespace vr {
namespace {

// ----------------------------------------------------------------------------------------------
// FP32 decision arithmetic: ray generation and slab clipping
// ----------------------------------------------------------------------------------------------
// Pixel (i, j)'s ray before the view rotation: the offset y = e - t of its origin from the
// view translation (y2 = 0 - t2 for both projections, so only y0, y1 vary per pixel) and its
// direction in world space.
__device__ __forceinline__ void ray_eye(const Cam &c, int i, int j, float &y0, float &y1, float d[3]) {
    float sx = __fsub_rn(__fmul_rn(__fdiv_rn(__fadd_rn((float)i, 0.5f), (float)c.W), 2.0f), 1.0f);
    float sy = __fsub_rn(1.0f, __fmul_rn(__fdiv_rn(__fadd_rn((float)j, 0.5f), (float)c.H), 2.0f));
    float e0, e1, de0, de1, de2;
    if (c.proj == 0) {
        e0 = __fmul_rn(sx, c.half_w);
        e1 = __fmul_rn(sy, c.half_h);
        de0 = 0.0f; de1 = 0.0f; de2 = -1.0f;
    } else {
        e0 = e1 = 0.0f;
        float x = __fmul_rn(sx, c.th_w), y = __fmul_rn(sy, c.th), z = -1.0f;
        float n2 = __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
        float len = __fsqrt_rn(n2);
        de0 = __fdiv_rn(x, len); de1 = __fdiv_rn(y, len); de2 = __fdiv_rn(z, len);
    }
    y0 = __fsub_rn(e0, c.t[0]);
    y1 = __fsub_rn(e1, c.t[1]);
#pragma unroll
    for (int k = 0; k < 3; ++k)     // world = R^T (eye - t)
        d[k] = __fadd_rn(__fadd_rn(__fmul_rn(c.R[k], de0), __fmul_rn(c.R[3 + k], de1)),
                         __fmul_rn(c.R[6 + k], de2));
}

// World coordinate k of the origin of a ray whose eye-space offset is (y0, y1, 0 - t2).
__device__ __forceinline__ float ray_origin(const Cam &c, int k, float y0, float y1) {
    const float y2 = __fsub_rn(0.0f, c.t[2]);
    return __fadd_rn(__fadd_rn(__fmul_rn(c.R[k], y0), __fmul_rn(c.R[3 + k], y1)), __fmul_rn(c.R[6 + k], y2));
}

__device__ __forceinline__ void ray_for_pixel(const Cam &c, int i, int j, float o[3], float d[3]) {
    float y0, y1;
    ray_eye(c, i, j, y0, y1, d);
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = ray_origin(c, k, y0, y1);
}

// Lattice range [k0, k1) of the samples inside the half-open box [lo, hi), t >= 0.
__device__ __forceinline__ bool box_krange(const float o[3], const float d[3], const float lo[3],
                                           const float hi[3], float step, int &k0, int &k1) {
    float tin = 0.0f, tout = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (!(lo[a] <= o[a] && o[a] < hi[a])) return false;
        } else {
            float t0 = __fdiv_rn(__fsub_rn(lo[a], o[a]), d[a]);
            float t1 = __fdiv_rn(__fsub_rn(hi[a], o[a]), d[a]);
            float en = t0 < t1 ? t0 : t1, ex = t0 < t1 ? t1 : t0;
            if (en > tin) tin = en;
            if (ex < tout) tout = ex;
        }
    }
    if (!(tout > tin) || !(tout < INFINITY)) return false;   // no direction: no samples
    k0 = (int)ceilf(__fdiv_rn(tin, step));
    k1 = (int)ceilf(__fdiv_rn(tout, step));
    return k1 > k0;
}

// Local stored coordinate of sample k along one axis, x = o + (k*step)*d - c, evaluated with
// error-free transformations (two-sum, fma residuals) and rounded once, so the anchor is
// accurate to half an ulp of a brick-local coordinate even when t is thousands of voxels.
__device__ __forceinline__ float anchor(float o, float d, float c, int k, float step) {
    float kf = (float)k;
    float th = __fmul_rn(kf, step);
    float tl = __fmaf_rn(kf, step, -th);          // k*step = th + tl exactly
    float ph = __fmul_rn(th, d);
    float pl = __fmaf_rn(th, d, -ph);             // th*d = ph + pl exactly
    float s = __fsub_rn(o, c);                    // two-sum of o and -c
    float bb = __fsub_rn(s, o);
    float sl = __fadd_rn(__fsub_rn(o, __fsub_rn(s, bb)), __fsub_rn(-c, bb));
    float r = __fadd_rn(s, ph);                   // two-sum of s and ph
    float rb = __fsub_rn(r, s);
    float rl = __fadd_rn(__fsub_rn(s, __fsub_rn(r, rb)), __fsub_rn(ph, rb));
    float lo = __fadd_rn(__fadd_rn(rl, sl), __fadd_rn(pl, __fmul_rn(tl, d)));
    return __fadd_rn(r, lo);
}

template <int S>
__device__ __forceinline__ float ldv(const void *p, int i);
template <>
__device__ __forceinline__ float ldv<0>(const void *p, int i) { return __ldg(static_cast<const float *>(p) + i); }
template <>
__device__ __forceinline__ float ldv<1>(const void *p, int i) {
    return __half2float(__ldg(static_cast<const __half *>(p) + i));
}
template <>
__device__ __forceinline__ float ldv<2>(const void *p, int i) {
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(p) + i));
}

__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fadd_rn(a, __fmul_rn(f, __fsub_rn(b, a)));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// One DVR sample: trilinear value at local stored coordinate (x, y, z), table lookup.  Every
// operation is an explicit intrinsic (no contraction), so the forward kernel and the adjoint's
// replay of a ray produce bit-identical values.
struct DvrSample {
    int ix, iy, iz;         // lower stencil corner (stored indices)
    float fx, fy, fz;       // trilinear fractions
    float u;                // unclamped table coordinate (v - vmin) / (vmax - vmin)
    int li;                 // table interval
    float lf;               // fraction inside the interval
    float4 L0, D;           // the interval's first entry and the difference to the next
    float r, g, b, a;       // interpolated colour and opacity
};

// Cell of a sample: lower stencil corner (local stored index, clamped so the 2x2x2 stencil stays
// inside the stored brick) and the trilinear fractions.
struct Cell {
    int ix, iy, iz;
    float fx, fy, fz;
};

// floor(x) as a float and as an int, for |x| < 2^22, on the FMA and integer pipes (floorf and
// float <-> int conversions issue on the narrower conversion pipe, which the per-sample work
// kept a third busy): x + 1.5 * 2^23 rounded toward -infinity lands on the float grid of
// spacing 1, exactly at floor(x) + 1.5 * 2^23, so the difference is exact and the integer sits in
// the low mantissa bits.  (For x = -0 the float floor is +0 where floorf gives -0; the fraction
// x - floor is then -0 instead of +0: the same value.)
constexpr float kFloorMagic = 12582912.0f;          // 1.5 * 2^23
constexpr int kFloorMagicBits = 0x4B400000;         // its bit pattern
__device__ __forceinline__ int floor_split(float x, float &fl) {
    const float t = __fadd_rd(x, kFloorMagic);
    fl = __fsub_rn(t, kFloorMagic);
    return __float_as_int(t) - kFloorMagicBits;
}

// An int n with |n| < 2^22 as a float, exactly, without a conversion instruction.
__device__ __forceinline__ float small_int_float(int n) {
    return __fsub_rn(__int_as_float(kFloorMagicBits + n), kFloorMagic);
}

// Brick-local coordinates are below 2^17 in magnitude (stored bricks span at most 65536 + 2
// voxels per axis), well inside floor_split's range.
template <bool CLAMP = true>
__device__ __forceinline__ void cell_of(float x, float y, float z, int mx, int my, int mz, Cell &c) {
    float flx, fly, flz;
    const int jx = floor_split(x, flx), jy = floor_split(y, fly), jz = floor_split(z, flz);
    c.fx = __fsub_rn(x, flx); c.fy = __fsub_rn(y, fly); c.fz = __fsub_rn(z, flz);
    if (CLAMP) {
        c.ix = clampi(jx, 0, mx); c.iy = clampi(jy, 0, my); c.iz = clampi(jz, 0, mz);
    } else {                          // caller has shown every index of the segment is in range
        c.ix = jx; c.iy = jy; c.iz = jz;
    }
}

// Shared-memory slots (float4) of table entry i and of its difference to entry i + 1, n entries:
// all entries, then all differences.  16-byte strides put any 8 consecutive entries in 8
// different bank groups (interleaved pairs repeat every 4 entries: measurably more conflicts).
__device__ __forceinline__ int tab_entry(int i, int) { return i; }
__device__ __forceinline__ int tab_diff(int i, int n) { return n + i; }

// Trilinear value from the 8 corners v[x + 2y + 4z], then the table lookup.
__device__ __forceinline__ void interp_tf(const float v[8], const Cell &c, bool scaled, float scale,
                                          float vmin, float inv_range, float lutmax, int lmax,
                                          const float4 *s_lut, DvrSample &o) {
    o.fx = c.fx; o.fy = c.fy; o.fz = c.fz;
    const float a00 = __fmaf_rn(c.fx, __fsub_rn(v[1], v[0]), v[0]);
    const float a10 = __fmaf_rn(c.fx, __fsub_rn(v[3], v[2]), v[2]);
    const float a01 = __fmaf_rn(c.fx, __fsub_rn(v[5], v[4]), v[4]);
    const float a11 = __fmaf_rn(c.fx, __fsub_rn(v[7], v[6]), v[6]);
    const float b0 = __fmaf_rn(c.fy, __fsub_rn(a10, a00), a00);
    const float b1 = __fmaf_rn(c.fy, __fsub_rn(a11, a01), a01);
    float val = __fmaf_rn(c.fz, __fsub_rn(b1, b0), b0);
    if (scaled) val = __fmul_rn(val, scale);
    o.u = __fmul_rn(__fsub_rn(val, vmin), inv_range);
    const float uc = __saturatef(o.u);          // clamp to [0, 1] (one instruction)
    const float xl = __fmul_rn(uc, lutmax);    // in [0, lutmax]
    // x = n - 1 (u >= 1) takes entry n - 1 with fraction 0: its stored difference is 0, so the
    // colour is entry n - 1 itself and no clamp of the interval is needed
    float fl;
    o.li = floor_split(xl, fl);
    o.lf = __fsub_rn(xl, fl);
    o.L0 = s_lut[tab_entry(o.li, lmax + 2)];
    o.D = s_lut[tab_diff(o.li, lmax + 2)];
    o.r = __fmaf_rn(o.lf, o.D.x, o.L0.x);
    o.g = __fmaf_rn(o.lf, o.D.y, o.L0.y);
    o.b = __fmaf_rn(o.lf, o.D.z, o.L0.z);
    o.a = __fmaf_rn(o.lf, o.D.w, o.L0.w);
}

// The table in shared memory with its differences entry i+1 - entry i: the same IEEE
// subtractions a lookup would do, made once per block instead of once per sample.
__device__ __forceinline__ void load_table(const float4 *__restrict__ lut, int n, float4 *s) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 a = lut[i];
        const float4 b = i + 1 < n ? lut[i + 1] : a;
        s[tab_entry(i, n)] = a;
        s[tab_diff(i, n)] = make_float4(__fsub_rn(b.x, a.x), __fsub_rn(b.y, a.y), __fsub_rn(b.z, a.z),
                                   __fsub_rn(b.w, a.w));
    }
}

// Strides of x, y, z in the stored brick (its layout: any axis may be the contiguous one).
struct Strides {
    int x, y, z;
};

// A brick's slice atlas (see DrawBrick::atlas): where its stored slice z starts.
struct Atlas {
    unsigned long long tex;
    int alog, dx, dy;
};

// A BF16 code widened to binary32 (exact: the code is the top half of the float).
__device__ __forceinline__ float bf16_value(unsigned int c) { return __uint_as_float(c << 16); }

// The 2x2 footprint (ix..ix+1, iy..iy+1) of slice iz and of slice iz+1, two texture gathers.
// A gather at unnormalised (x, y) returns the texels at floor(x - 1/2) and the next one on
// each axis, ordered ((x0,y1), (x1,y1), (x1,y0), (x0,y0)); x = ix + 1 selects exactly ix.  The
// texels are returned unfiltered, so the corners are the stored values themselves.
template <int S>
__device__ __forceinline__ void fetch8_atlas(const Atlas &a, int ix, int iy, int iz, float v[8]) {
    const int cm = (1 << a.alog) - 1, col = iz & cm;   // atlas coordinates < 32768
    const float x0 = small_int_float(col * a.dx + ix + 1), y0 = small_int_float((iz >> a.alog) * a.dy + iy + 1);
    // slice iz + 1: the next tile of the row, or the first tile of the next row
    const bool wrap = col == cm;
    const float x1 = __fadd_rn(x0, small_int_float(wrap ? -cm * a.dx : a.dx));
    const float y1 = wrap ? __fadd_rn(y0, small_int_float(a.dy)) : y0;
    if constexpr (S != 2) {           // FP32 texels, or FP16 ones the texture unit widens (exactly)
        const float4 g0 = tex2Dgather<float4>(a.tex, x0, y0, 0);
        const float4 g1 = tex2Dgather<float4>(a.tex, x1, y1, 0);
        v[0] = g0.w; v[1] = g0.z; v[2] = g0.x; v[3] = g0.y;
        v[4] = g1.w; v[5] = g1.z; v[6] = g1.x; v[7] = g1.y;
    } else {                          // BF16 codes as 16-bit unsigned texels
        const uint4 g0 = tex2Dgather<uint4>(a.tex, x0, y0, 0);
        const uint4 g1 = tex2Dgather<uint4>(a.tex, x1, y1, 0);
        v[0] = bf16_value(g0.w); v[1] = bf16_value(g0.z);
        v[2] = bf16_value(g0.x); v[3] = bf16_value(g0.y);
        v[4] = bf16_value(g1.w); v[5] = bf16_value(g1.z);
        v[6] = bf16_value(g1.x); v[7] = bf16_value(g1.y);
    }
}

// A 16-bit code of a pair texel widened to binary32 (exact): FP16 through the half conversion,
// BF16 as the top half of the float.
template <int S>
__device__ __forceinline__ float code_value(unsigned int c) {
    if constexpr (S == 1) return __half2float(__ushort_as_half((unsigned short)c));
    else return bf16_value(c);
}

// Pair atlas (16-bit bricks): tile iz holds, in each 32-bit texel (x, y), the codes of voxel
// (x, y, iz) (low half) and (x, y, iz + 1) (high half), so one gather at slice iz's footprint
// returns all 8 stencil corners -- 16 bytes of texels per sample instead of 32, one gather
// instead of two.  Tiles are placed like the slice atlas's, one per slice but the last.
__device__ __forceinline__ uint4 gather_pair(const Atlas &a, int ix, int iy, int iz) {
    const int cm = (1 << a.alog) - 1;                   // atlas coordinates < 32768
    const float x0 = small_int_float((iz & cm) * a.dx + ix + 1), y0 = small_int_float((iz >> a.alog) * a.dy + iy + 1);
    return tex2Dgather<uint4>(a.tex, x0, y0, 0);
}

template <int S>
__device__ __forceinline__ void unpack_pair(const uint4 g, float v[8]) {
    v[0] = code_value<S>(g.w & 0xffffu); v[4] = code_value<S>(g.w >> 16);
    v[1] = code_value<S>(g.z & 0xffffu); v[5] = code_value<S>(g.z >> 16);
    v[2] = code_value<S>(g.x & 0xffffu); v[6] = code_value<S>(g.x >> 16);
    v[3] = code_value<S>(g.y & 0xffffu); v[7] = code_value<S>(g.y >> 16);
}

template <int S>
__device__ __forceinline__ void fetch8_pair(const Atlas &a, int ix, int iy, int iz, float v[8]) {
    unpack_pair<S>(gather_pair(a, ix, iy, iz), v);
}

// Whether fetch mode F reads a texture (the slice atlas, 2, or the pair atlas, 5).
constexpr bool gathers(int F) { return F == 2 || F == 5; }

template <int S>
__device__ __forceinline__ void fetch8(const void *src, int i0, const Strides &t, float v[8]) {
    v[0] = ldv<S>(src, i0);             v[1] = ldv<S>(src, i0 + t.x);
    v[2] = ldv<S>(src, i0 + t.y);       v[3] = ldv<S>(src, i0 + t.y + t.x);
    v[4] = ldv<S>(src, i0 + t.z);       v[5] = ldv<S>(src, i0 + t.z + t.x);
    v[6] = ldv<S>(src, i0 + t.z + t.y); v[7] = ldv<S>(src, i0 + t.z + t.y + t.x);
}

// Disabled spectral channels hold vmin (the bottom of the table range) in place of their data:
// the stencil's two z-planes are global channels org_z + iz and + 1 (clamped at the cube
// border, like the ghost copies).  `vcode` is vmin in the brick's stored units.
__device__ __forceinline__ void mask_channels(float v[8], int iz, int org_z, int nz,
                                              const unsigned char *chmask, float vcode) {
    const int z0 = clampi(org_z + iz, 0, nz - 1), z1 = clampi(org_z + iz + 1, 0, nz - 1);
    if (!chmask[z0]) { v[0] = vcode; v[1] = vcode; v[2] = vcode; v[3] = vcode; }
    if (!chmask[z1]) { v[4] = vcode; v[5] = vcode; v[6] = vcode; v[7] = vcode; }
}

template <int S>
__device__ __forceinline__ void dvr_sample(const void *src, const Strides &t, int mx, int my, int mz,
                                           float scale, float x, float y, float z, float vmin,
                                           float inv_range, float lutmax, int lmax,
                                           const float4 *s_lut, const unsigned char *chmask,
                                           int org_z, int nz, float vcode, DvrSample &o,
                                           const Atlas *atl = nullptr) {
    Cell c;
    cell_of(x, y, z, mx, my, mz, c);
    o.ix = c.ix; o.iy = c.iy; o.iz = c.iz;
    float v[8];
    if (atl)                          // the same texels from the brick's slice atlas
        fetch8_atlas<S>(*atl, c.ix, c.iy, c.iz, v);
    else
        fetch8<S>(src, c.ix * t.x + c.iy * t.y + c.iz * t.z, t, v);
    if (chmask) mask_channels(v, c.iz, org_z, nz, chmask, vcode);
    interp_tf(v, c, S != 0, scale, vmin, inv_range, lutmax, lmax, s_lut, o);
}

// Stencil cache of one ray: the 8 corner values of the previous sample's cell.  Moving to an
// adjacent cell (each index changes by at most 1) keeps the corners the two cells share and
// gathers only the others; any larger jump reloads all 8.  `need` bit c marks corner c as
// still to be gathered; shifting the values shifts their bits too.
template <int S>
__device__ __forceinline__ void fetch8_cached(const void *src, const Strides &t, const Cell &c,
                                              int &px, int &py, int &pz, float v[8]) {
    const int ddx = c.ix - px, ddy = c.iy - py, ddz = c.iz - pz;
    unsigned need = 0u;
    if (ddx < -1 || ddx > 1 || ddy < -1 || ddy > 1 || ddz < -1 || ddz > 1) {
        need = 0xffu;
    } else {
        if (ddx == 1) {
            v[0] = v[1]; v[2] = v[3]; v[4] = v[5]; v[6] = v[7];
            need = ((need >> 1) & 0x55u) | 0xaau;
        } else if (ddx == -1) {
            v[1] = v[0]; v[3] = v[2]; v[5] = v[4]; v[7] = v[6];
            need = ((need << 1) & 0xaau) | 0x55u;
        }
        if (ddy == 1) {
            v[0] = v[2]; v[1] = v[3]; v[4] = v[6]; v[5] = v[7];
            need = ((need >> 2) & 0x33u) | 0xccu;
        } else if (ddy == -1) {
            v[2] = v[0]; v[3] = v[1]; v[6] = v[4]; v[7] = v[5];
            need = ((need << 2) & 0xccu) | 0x33u;
        }
        if (ddz == 1) {
            v[0] = v[4]; v[1] = v[5]; v[2] = v[6]; v[3] = v[7];
            need = ((need >> 4) & 0x0fu) | 0xf0u;
        } else if (ddz == -1) {
            v[4] = v[0]; v[5] = v[1]; v[6] = v[2]; v[7] = v[3];
            need = ((need << 4) & 0xf0u) | 0x0fu;
        }
    }
    px = c.ix; py = c.iy; pz = c.iz;
    const int i0 = c.ix * t.x + c.iy * t.y + c.iz * t.z;
    if (need & 0x01u) v[0] = ldv<S>(src, i0);
    if (need & 0x02u) v[1] = ldv<S>(src, i0 + t.x);
    if (need & 0x04u) v[2] = ldv<S>(src, i0 + t.y);
    if (need & 0x08u) v[3] = ldv<S>(src, i0 + t.y + t.x);
    if (need & 0x10u) v[4] = ldv<S>(src, i0 + t.z);
    if (need & 0x20u) v[5] = ldv<S>(src, i0 + t.z + t.x);
    if (need & 0x40u) v[6] = ldv<S>(src, i0 + t.z + t.y);
    if (need & 0x80u) v[7] = ldv<S>(src, i0 + t.z + t.y + t.x);
}

// Front-to-back "over" of one sample into (c, T): c += T a rgb, T *= 1 - a.
__device__ __forceinline__ void over(const DvrSample &s, float &c0, float &c1, float &c2, float &T) {
    const float w = __fmul_rn(T, s.a);
    c0 = __fmaf_rn(w, s.r, c0);
    c1 = __fmaf_rn(w, s.g, c1);
    c2 = __fmaf_rn(w, s.b, c2);
    T = __fmaf_rn(-T, s.a, T);                 // T (1 - a), one rounding
}

// ----------------------------------------------------------------------------------------------
// ray cast: one CTA = 32x8 (or 8x32) pixels of one brick's rendering rectangle; warp = 32 pixels
// along the image axis that the brick layout follows
// ----------------------------------------------------------------------------------------------
// One brick segment of a ray: n lattice samples from the anchor q, composited front to back
// until the segment's transmittance reaches the threshold.  Returns the samples composited.
// F: how the stencil is read (FrameConsts::fetch).  MASK: a spectral-channel mask is set (its own
// instantiation, so unmasked frames carry none of its registers or branches).
// The segment loop over a pair atlas, software-pipelined: a sample is one gather, so the gather
// of sample j + 1 is issued before sample j is interpolated and composited (its latency overlaps
// that work at the cost of one more texel quad in registers).  Samples, their order and the
// arithmetic are those of the plain loop.
template <int S, bool CLAMP, bool MASK>
__device__ __forceinline__ int dvr_segment_pair(const Atlas &atl, int mx, int my, int mz, float scale,
                                                float qx, float qy, float qz, const float d[3], int n,
                                                const FrameConsts &fc, const float4 *s_lut, int org_z, float vcode,
                                                float &c0, float &c1, float &c2, float &T) {
    const float vmin = fc.vmin, inv_range = fc.inv_range, lutmax = fc.lutmax, thr = fc.thr;
    const int lmax = fc.nlut - 2;
    const float nf = (float)n;            // exact: n <= 2^24 + 1, checked by the host
    if (n <= 0) return 0;
    Cell cl;
    cell_of<CLAMP>(qx, qy, qz, mx, my, mz, cl);
    uint4 g = gather_pair(atl, cl.ix, cl.iy, cl.iz);
    float jf = 0.0f;
    for (;;) {
        const float jn = __fadd_rn(jf, 1.0f);
        Cell cn;
        uint4 gn = make_uint4(0u, 0u, 0u, 0u);
        if (jn < nf) {                    // the next sample's cell and gather, ahead
            const float tn = __fmul_rn(jn, fc.step);
            cell_of<CLAMP>(__fmaf_rn(tn, d[0], qx), __fmaf_rn(tn, d[1], qy), __fmaf_rn(tn, d[2], qz),
                           mx, my, mz, cn);
            gn = gather_pair(atl, cn.ix, cn.iy, cn.iz);
        }
        float v[8];
        unpack_pair<S>(g, v);
        if (MASK) mask_channels(v, cl.iz, org_z, fc.nz, fc.chmask, vcode);
        DvrSample sm;
        interp_tf(v, cl, S != 0, scale, vmin, inv_range, lutmax, lmax, s_lut, sm);
        over(sm, c0, c1, c2, T);
        if (T <= thr) return (int)jf + 1;
        if (!(jn < nf)) return (int)jn;
        jf = jn;
        cl = cn;
        g = gn;
    }
}

template <int S, int F, bool CLAMP, bool MASK, bool ICOUNT = false>
__device__ __forceinline__ int dvr_segment(const void *src, const Strides &st, const Atlas &atl,
                                           int mx, int my, int mz,
                                           float scale, float qx, float qy, float qz, const float d[3],
                                           int n, const FrameConsts &fc, const float4 *s_lut,
                                           int org_z, float vcode,
                                           float &c0, float &c1, float &c2, float &T) {
    if constexpr (F == 5 && VR_PAIR_PIPELINE)
        return dvr_segment_pair<S, CLAMP, MASK>(atl, mx, my, mz, scale, qx, qy, qz, d, n, fc, s_lut, org_z, vcode,
                                                c0, c1, c2, T);
    const float vmin = fc.vmin, inv_range = fc.inv_range, lutmax = fc.lutmax, thr = fc.thr;
    const int lmax = fc.nlut - 2;
    int px = -4, py = -4, pz = -4;        // no cell cached yet
    float v[8];
    // the sample index as a float (exact: n <= 2^24 + 1, checked by the host), and as an int
    // beside it where that takes fewer registers (ICOUNT)
    const float nf = (float)n;
    float jf = 0.0f;
    int j = 0;
#pragma unroll kSampleUnroll
    for (; ICOUNT ? j < n : jf < nf; ++j, jf = __fadd_rn(jf, 1.0f)) {
        const float tj = __fmul_rn(jf, fc.step);
        Cell cl;
        cell_of<CLAMP>(__fmaf_rn(tj, d[0], qx), __fmaf_rn(tj, d[1], qy), __fmaf_rn(tj, d[2], qz),
                       mx, my, mz, cl);
        if (F == 2)
            fetch8_atlas<S>(atl, cl.ix, cl.iy, cl.iz, v);
        else if (F == 5)
            fetch8_pair<S>(atl, cl.ix, cl.iy, cl.iz, v);
        else if (F == 1)
            fetch8_cached<S>(src, st, cl, px, py, pz, v);
        else
            fetch8<S>(src, cl.ix * st.x + cl.iy * st.y + cl.iz * st.z, st, v);
        if (MASK) mask_channels(v, cl.iz, org_z, fc.nz, fc.chmask, vcode);
        DvrSample sm;
        interp_tf(v, cl, S != 0, scale, vmin, inv_range, lutmax, lmax, s_lut, sm);
        over(sm, c0, c1, c2, T);
        if (T <= thr) return (ICOUNT ? j : (int)jf) + 1;
    }
    return ICOUNT ? j : (int)jf;
}

// F = 1: a ray keeps the stencil corners its next cell shares with the last one (fewer loads,
// more instructions; pays off when a warp's loads scatter over many cache lines); F = 0: all
// eight corners are loaded for every sample; F = 2: two gathers from the slice atlas.
// MODE 0: DVR, one fragment (colour, transmittance) per (brick, pixel of its rectangle);
// MODE 1: MIP, one maximum per (brick, pixel).
// Pixel (rx, ry) of a work item's rectangle that lane `lane` of warp `w` (0..7) ray-casts:
// lanes 0: a warp is 32 pixels along image x (tile 32x8); 1: along image y (tile 8x32).  (Warps
// of 8x4 pixels in 2x2 quads, for texture-quad locality, measured 10 % slower.)
__device__ __forceinline__ void thread_pixel(int lanes, const TileItem &it, int w, int lane, int &rx, int &ry) {
    if (lanes == 1) {
        rx = it.tx * kRcShort + w;
        ry = it.ty * kRcLong + lane;
    } else {
        rx = it.tx * kRcLong + lane;
        ry = it.ty * kRcShort + w;
    }
}

// The 32 rays of one warp: strip `strip` (0..7) of work item `it`; writes their fragments and
// adds the warp's samples to the counters.
template <int S, int MODE, int F, bool MASK>
__device__ __forceinline__ void rc_strip(const FrameConsts &fc, const float4 *__restrict__ lut,
                                         DrawBrick *__restrict__ dbs, const TileItem it, int strip, int lane,
                                         const void *__restrict__ pool, void *__restrict__ frags,
                                         Counters *__restrict__ ctr, float4 *s_lut) {
    const DrawBrick &b = dbs[it.db];
    // a warp's 32 rays are adjacent pixels along the image axis the brick layout follows
    int rx, ry;
    thread_pixel(fc.lanes_y, it, strip, lane, rx, ry);
    const int rw = b.rect[2];
    const bool inrect = rx < rw && ry < b.rect[3];
    int nsamp = 0;
    float o[3], d[3];
    int k0 = 0, k1 = 0;
    bool hit = false;
    if (inrect) {
        ray_for_pixel(fc.cam, b.rect[0] + rx, b.rect[1] + ry, o, d);
        hit = box_krange(o, d, b.lo, b.hi, fc.step, k0, k1);
    }
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
    if (inrect) {
        const long long fi = b.frag_off + (long long)ry * rw + rx;
        const void *src = static_cast<const char *>(pool) +
                          b.data_off * (S == 0 ? 4 : 2);
        const Strides st{b.str[0], b.str[1], b.str[2]};
        const int mx = b.dim[0] - 2, my = b.dim[1] - 2, mz = b.dim[2] - 2;
        const float scale = S == 0 ? 1.0f : ldexpf(1.0f, b.exp2);
        const Atlas atl{gathers(F) ? b.atlas : 0ull, b.alog, b.dim[0], b.dim[1]};
        if (MODE == 0) {
            if (hit) {
                const float qx = anchor(o[0], d[0], b.org_c[0], k0, fc.step);
                const float qy = anchor(o[1], d[1], b.org_c[1], k0, fc.step);
                const float qz = anchor(o[2], d[2], b.org_c[2], k0, fc.step);
                const int n = k1 - k0;
                // sample positions are monotone along the ray: when the segment's first and last
                // cells are inside the stored brick, every cell in between is too
                Cell e0, e1;
                const float tl = __fmul_rn((float)(n - 1), fc.step);
                cell_of<false>(qx, qy, qz, mx, my, mz, e0);
                cell_of<false>(__fmaf_rn(tl, d[0], qx), __fmaf_rn(tl, d[1], qy), __fmaf_rn(tl, d[2], qz),
                               mx, my, mz, e1);
                const bool inside = min(e0.ix, e1.ix) >= 0 && max(e0.ix, e1.ix) <= mx &&
                                    min(e0.iy, e1.iy) >= 0 && max(e0.iy, e1.iy) <= my &&
                                    min(e0.iz, e1.iz) >= 0 && max(e0.iz, e1.iz) <= mz;
                const float vcode = S == 0 ? fc.vmin : ldexpf(fc.vmin, -b.exp2);
                constexpr bool icount = MASK && S == 2;      // BF16 masked: an int count spills less
                const int j = inside
                    ? dvr_segment<S, F, false, MASK, icount>(src, st, atl, mx, my, mz, scale, qx, qy, qz, d, n, fc,
                                                             s_lut, b.org[2], vcode, c0, c1, c2, T)
                    : dvr_segment<S, F, true, MASK, icount>(src, st, atl, mx, my, mz, scale, qx, qy, qz, d, n, fc,
                                                            s_lut, b.org[2], vcode, c0, c1, c2, T);
                nsamp = j;
            }
            static_cast<float4 *>(frags)[fi] = make_float4(c0, c1, c2, T);   // .w = transmittance
        } else {
            float m = -INFINITY;
            if (hit) {
                for (int k = k0; k < k1; ++k) {
                    const float t = __fmul_rn((float)k, fc.step);
                    const float px = __fadd_rn(o[0], __fmul_rn(t, d[0]));
                    const float py = __fadd_rn(o[1], __fmul_rn(t, d[1]));
                    const float pz = __fadd_rn(o[2], __fmul_rn(t, d[2]));
                    const float x = __fsub_rn(px, 0.5f), y = __fsub_rn(py, 0.5f), z = __fsub_rn(pz, 0.5f);
                    // floors on the FMA and integer pipes (world coordinates are far below 2^22)
                    float flx, fly, flz;
                    const int jx = floor_split(x, flx), jy = floor_split(y, fly), jz = floor_split(z, flz);
                    const float fx = __fsub_rn(x, flx), fy = __fsub_rn(y, fly), fz = __fsub_rn(z, flz);
                    const int ix = clampi(jx - b.org[0], 0, mx);
                    const int iy = clampi(jy - b.org[1], 0, my);
                    const int iz = clampi(jz - b.org[2], 0, mz);
                    const int i0 = ix * st.x + iy * st.y + iz * st.z;
                    float v[8];
                    if (F == 2)
                        fetch8_atlas<S>(atl, ix, iy, iz, v);
                    else if (F == 5)
                        fetch8_pair<S>(atl, ix, iy, iz, v);
                    else
                        fetch8<S>(src, i0, st, v);
                    if (MASK)
                        mask_channels(v, iz, b.org[2], fc.nz, fc.chmask,
                                      S == 0 ? fc.vmin : ldexpf(fc.vmin, -b.exp2));
                    const float c00 = lerp_rn(v[0], v[1], fx);
                    const float c10 = lerp_rn(v[2], v[3], fx);
                    const float c01 = lerp_rn(v[4], v[5], fx);
                    const float c11 = lerp_rn(v[6], v[7], fx);
                    float val = lerp_rn(lerp_rn(c00, c10, fy), lerp_rn(c01, c11, fy), fz);
                    if (S != 0) val = __fmul_rn(val, scale);
                    m = val > m ? val : m;
                }
                nsamp = k1 - k0;
            }
            static_cast<float *>(frags)[fi] = m;
        }
    }
    const unsigned int tot = __reduce_add_sync(0xffffffffu, (unsigned int)nsamp);
    if (lane == 0 && tot > 0) {
        atomicAdd(&ctr->samples, (unsigned long long)tot);
        if (atomicExch(&dbs[it.db].sampled, 1) == 0) {
            atomicAdd(&ctr->bricks_sampled, 1ull);
            atomicAdd(&ctr->brick_bytes_sampled, (unsigned long long)b.bytes);
        }
    }
}

// Blocks per SM the registers of k_raycast<., MODE, F, .> must allow (1: no constraint beyond
// one block): the kernel's speed follows its resident warps, and 40 registers (6 CTAs) hold the
// atlas DVR loop without spills.
template <int MODE, int F>
constexpr int rc_min_blocks() {
    return MODE == 0 ? (gathers(F) && VR_DVR_MIN_BLOCKS > 0 ? VR_DVR_MIN_BLOCKS : 1)
                     : (VR_MIP_MIN_BLOCKS > 0 ? VR_MIP_MIN_BLOCKS : 1);
}

template <int S, int MODE, int F, bool MASK>
__global__ void __launch_bounds__(256, rc_min_blocks<MODE, F>())
k_raycast(const FrameConsts fc, const float4 *__restrict__ lut, DrawBrick *__restrict__ dbs,
          const TileItem *__restrict__ items, const void *__restrict__ pool, void *__restrict__ frags,
          Counters *__restrict__ ctr) {
    extern __shared__ float4 s_lut[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (MODE == 0) {
        load_table(lut, fc.nlut, s_lut);
        __syncthreads();
    }
    rc_strip<S, MODE, F, MASK>(fc, lut, dbs, items[blockIdx.x], warp, lane, pool, frags, ctr, s_lut);
}

// ----------------------------------------------------------------------------------------------
// staged ray cast (fetch 4): the rays of a work item cross their brick along its march axis M (the
// view's dominant axis other than the contiguous axis L of the brick copy); the block walks that
// axis in chunks of kStageC lower-stencil indices, copies each chunk's slab of the brick -- the
// bounding box of the tile's four corner rays across the chunk, widened by the stencil and a
// margin -- into shared memory with one bulk copy per row of the padded copy, one chunk ahead
// (two stages, an mbarrier each), and samples the stencils from there.  Each ray processes its
// samples in order, stopping at a chunk's end; a stencil outside the staged slab (or a chunk
// whose slab does not fit a stage, or a ray crossing M the other way) is read from global
// memory instead, so every sample and every frame is exactly the linear path's.
// ----------------------------------------------------------------------------------------------
constexpr int kStageC = 8;              // lower-stencil indices per chunk along the march axis
constexpr int kStageFloats = 7168;      // floats per stage (28 KB)
constexpr int kStageSpin = 1 << 21;     // bound of a wait for a stage's copies (polls ~32 ns apart:
                                        // ~0.1 s, against microseconds for a slab)

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Whether the phase of `bar` with parity `parity` has completed (no blocking).
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// One row of the slab: `bytes` (a multiple of 16) from 16-byte-aligned global `src` to
// 16-byte-aligned shared `dst`, counted on `bar`.
__device__ __forceinline__ void bulk_row(float *dst, const float *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// The slab a stage holds: stored-brick index ranges [lo, lo + n) per world axis, the floats per
// shared row (its contiguous-axis extent, a multiple of 4) and the stage's bytes (0: nothing
// staged; the chunk's stencils are read from global memory).
struct StageBox {
    int lo[3], n[3];
    int row, bytes;
};

// Element a of a three-element register array by selects (a dynamic index would put the
// array in local memory).
__device__ __forceinline__ float pick3(const float v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }
__device__ __forceinline__ int pick3(const int v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

// Warp 0: the slab of chunk c (march-axis lower indices [c C, c C + C)) from the tile's four corner
// rays, and its bulk copies into stage s.  Every lane takes a corner (lane & 3); lane 0 arms the
// stage's barrier with the slab's bytes before any lane issues a row.
__device__ __forceinline__ void stage_slab(const FrameConsts &fc, const DrawBrick &b, const TileItem &it, int M,
                                           int L, int O, int c, int s, float *stage, const float *__restrict__ pool,
                                           StageBox *box, unsigned long long *bar, bool off) {
    const int lane = threadIdx.x & 31;
    // the tile's pixel range inside the rectangle
    const int tw = fc.lanes_y ? kRcShort : kRcLong, th = fc.lanes_y ? kRcLong : kRcShort;
    const int px0 = it.tx * tw, py0 = it.ty * th;
    const int px1 = min(px0 + tw, b.rect[2]) - 1, py1 = min(py0 + th, b.rect[3]) - 1;
    const int cx = (lane & 1) ? px1 : px0, cy = (lane & 2) ? py1 : py0;
    float o[3], d[3];
    ray_for_pixel(fc.cam, b.rect[0] + cx, b.rect[1] + cy, o, d);
    const int dimM = b.dim[M], dimL = b.dim[L], dimO = b.dim[O];
    const int m0 = c * kStageC;
    int lo_l = 0x7fffffff, hi_l = -0x7fffffff, lo_o = 0x7fffffff, hi_o = -0x7fffffff;
    const float oM = pick3(o, M), dM = pick3(d, M), oL = pick3(o, L), dL = pick3(d, L), oO = pick3(o, O),
                dO = pick3(d, O);
    bool ok = dM != 0.0f;
    for (int e = 0; e < 2 && ok; ++e) {
        // the plane x_M = m0 (or m0 + C) of stored coordinates: x = p - org_c
        const float v = (float)(m0 + e * kStageC) + b.org_c[M];
        const float t = (v - oM) / dM;
        ok = t >= 0.0f;
        const float xl = fmaf(t, dL, oL) - b.org_c[L], xo = fmaf(t, dO, oO) - b.org_c[O];
        const int fl = (int)floorf(xl), fo = (int)floorf(xo);
        lo_l = min(lo_l, fl); hi_l = max(hi_l, fl);
        lo_o = min(lo_o, fo); hi_o = max(hi_o, fo);
    }
#pragma unroll
    for (int sh = 1; sh < 4; sh <<= 1) {
        lo_l = min(lo_l, __shfl_xor_sync(0xffffffffu, lo_l, sh));
        hi_l = max(hi_l, __shfl_xor_sync(0xffffffffu, hi_l, sh));
        lo_o = min(lo_o, __shfl_xor_sync(0xffffffffu, lo_o, sh));
        hi_o = max(hi_o, __shfl_xor_sync(0xffffffffu, hi_o, sh));
    }
    ok = __all_sync(0xffffffffu, ok) && !off && b.pad_off >= 0 && (unsigned)m0 <= (unsigned)(dimM - 1);
    // the stencil's upper neighbour and a margin of one voxel for rounding, inside the brick;
    // the contiguous axis from a 16-byte boundary, whole 16-byte pieces, within the padded row
    const int prow = (dimL + 3) & ~3;
    int l0 = max(lo_l - 1, 0) & ~3;
    int l1 = min(hi_l + 2, dimL - 1);
    int o0 = max(lo_o - 1, 0), o1 = min(hi_o + 2, dimO - 1);
    const int nm = min(kStageC + 1, dimM - m0);
    int row = ((l1 - l0 + 1) + 3) & ~3;
    if (l0 + row > prow) row = prow - l0;
    const int no = o1 - o0 + 1;
    long long floats = (long long)nm * no * row;
    // a stencil needs two indices along every axis of the slab
    if (!ok || l1 < l0 + 1 || o1 < o0 + 1 || nm < 2 || row < 4 || floats > kStageFloats) floats = 0;
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            box->lo[a] = a == L ? l0 : (a == O ? o0 : m0);
            box->n[a] = a == L ? row : (a == O ? no : nm);
        }
        box->row = row;
        box->bytes = (int)(floats * 4);
        if (floats > 0) mbar_expect_tx(bar, (unsigned)(floats * 4));
    }
    __syncwarp();
    if (floats == 0) return;
    const float *base = pool + b.pad_off + (long long)l0;
    const int sM = b.pad_str[M], sO = b.pad_str[O];
    for (int mi = 0; mi < nm; ++mi)
        for (int oi = lane; oi < no; oi += 32)
            bulk_row(stage + ((long long)mi * no + oi) * row,
                     base + (long long)(m0 + mi) * sM + (long long)(o0 + oi) * sO, (unsigned)(row * 4), bar);
}

template <bool MASK>
__global__ void __launch_bounds__(256, 3)
k_raycast_staged(const FrameConsts fc, const float4 *__restrict__ lut, DrawBrick *__restrict__ dbs,
                 const TileItem *__restrict__ items, const float *__restrict__ pool, float4 *__restrict__ frags,
                 Counters *__restrict__ ctr) {
    extern __shared__ float4 s_lut[];
    float *stages = reinterpret_cast<float *>(s_lut + 2 * fc.nlut);      // 2 x kStageFloats
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ StageBox s_box[2];
    __shared__ int s_rng[2][8];
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    load_table(lut, fc.nlut, s_lut);
    if (tid == 0) {
        mbar_init(&s_bar[0]);
        mbar_init(&s_bar[1]);
        mbar_fence_init();
        s_err = 0;
    }
    const TileItem it = items[blockIdx.x];
    DrawBrick &b = dbs[it.db];
    const int L = b.pad_str[0] == 1 ? 0 : (b.pad_str[1] == 1 ? 1 : 2);
    const int M = fc.stage_m, O = 3 - L - M;
    int rx, ry;
    thread_pixel(fc.lanes_y, it, warp, lane, rx, ry);
    const int rw = b.rect[2];
    const bool inrect = rx < rw && ry < b.rect[3];
    float o[3], d[3];
    int k0 = 0, k1 = 0;
    bool hit = false;
    if (inrect) {
        ray_for_pixel(fc.cam, b.rect[0] + rx, b.rect[1] + ry, o, d);
        hit = box_krange(o, d, b.lo, b.hi, fc.step, k0, k1);
    }
    const int mx = b.dim[0] - 2, my = b.dim[1] - 2, mz = b.dim[2] - 2;
    const int mM = b.dim[M] - 2;
    float q[3] = {0.0f, 0.0f, 0.0f};
    int n = 0;
    if (hit) {
        q[0] = anchor(o[0], d[0], b.org_c[0], k0, fc.step);
        q[1] = anchor(o[1], d[1], b.org_c[1], k0, fc.step);
        q[2] = anchor(o[2], d[2], b.org_c[2], k0, fc.step);
        n = k1 - k0;
    }
    const float dM = M == 0 ? d[0] : (M == 1 ? d[1] : d[2]);
    const float qM = M == 0 ? q[0] : (M == 1 ? q[1] : q[2]);
    const bool staged = hit && (fc.stage_dir > 0 ? dM > 0.2f : dM < -0.2f) && b.pad_off >= 0;
    // chunks of the ray's first and last samples (the loop's own position arithmetic)
    int cmin = 0x7fffffff, cmax = -1;
    if (staged) {
        const float tl = __fmul_rn((float)(n - 1), fc.step);
        float fl;
        const int i0 = clampi(floor_split(qM, fl), 0, mM);
        const int i1 = clampi(floor_split(__fmaf_rn(tl, dM, qM), fl), 0, mM);
        cmin = min(i0, i1) / kStageC;
        cmax = max(i0, i1) / kStageC;
    }
    for (int sh = 16; sh > 0; sh >>= 1) {
        cmin = min(cmin, __shfl_xor_sync(0xffffffffu, cmin, sh));
        cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, sh));
    }
    if (lane == 0) { s_rng[0][warp] = cmin; s_rng[1][warp] = cmax; }
    __syncthreads();                    // table, barriers and the warps' chunk ranges
    cmin = s_rng[0][0]; cmax = s_rng[1][0];
#pragma unroll
    for (int w = 1; w < 8; ++w) { cmin = min(cmin, s_rng[0][w]); cmax = max(cmax, s_rng[1][w]); }

    const float *src = pool + (b.pad_off >= 0 ? b.pad_off : b.data_off);
    const Strides gst = b.pad_off >= 0 ? Strides{b.pad_str[0], b.pad_str[1], b.pad_str[2]}
                                       : Strides{b.str[0], b.str[1], b.str[2]};
    const float vmin = fc.vmin, inv_range = fc.inv_range, lutmax = fc.lutmax, thr = fc.thr;
    const int lmax = fc.nlut - 2;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
    int j = 0;
    bool done = !hit;
    if (hit && !staged) {               // every stencil of this ray from global memory
        j = dvr_segment<0, 0, true, MASK>(src, gst, Atlas{0ull, 0, 0, 0}, mx, my, mz, 1.0f, q[0], q[1], q[2], d,
                                          n, fc, s_lut, b.org[2], fc.vmin, c0, c1, c2, T);
        done = true;
    }
    if (cmax >= cmin) {
        const int nch = cmax - cmin + 1;
        const int cbeg = fc.stage_dir > 0 ? cmin : cmax;
        unsigned phases = 0u;           // bit s: the parity stage s waits for next
        if (warp == 0) stage_slab(fc, b, it, M, L, O, cbeg, 0, stages, pool, &s_box[0], &s_bar[0], false);
        __syncthreads();
        for (int i = 0; i < nch; ++i) {
            const int cs = i & 1, c = cbeg + i * fc.stage_dir;
            if (i + 1 < nch && warp == 0)
                stage_slab(fc, b, it, M, L, O, c + fc.stage_dir, cs ^ 1, stages + (cs ^ 1) * kStageFloats, pool,
                           &s_box[cs ^ 1], &s_bar[cs ^ 1], s_err != 0);
            StageBox bx = s_box[cs];
            if (bx.bytes > 0) {         // this chunk's slab has landed
                bool ok = false;
                const unsigned par = (phases >> cs) & 1u;
                for (int r = 0; r < kStageSpin && !ok; ++r) {
                    ok = mbar_test_wait(&s_bar[cs], par);
                    if (!ok) __nanosleep(32);
                }
                phases ^= 1u << cs;
                if (!ok) {
                    s_err = 1;
                    atomicOr(reinterpret_cast<unsigned int *>(&ctr->pad), 1u);
                    bx.bytes = 0;
                }
            }
            const float *stage = stages + cs * kStageFloats;
            int so[3];                  // shared-memory strides of the slab by world axis
#pragma unroll
            for (int a = 0; a < 3; ++a) so[a] = a == L ? 1 : (a == O ? bx.row : bx.row * pick3(bx.n, O));
            const int mlo = c * kStageC, mhi = mlo + kStageC;
            float jf = (float)j;
            while (staged && !done && j < n) {
                const float tj = __fmul_rn(jf, fc.step);
                Cell cl;
                cell_of<true>(__fmaf_rn(tj, d[0], q[0]), __fmaf_rn(tj, d[1], q[1]), __fmaf_rn(tj, d[2], q[2]),
                              mx, my, mz, cl);
                const int im = M == 0 ? cl.ix : (M == 1 ? cl.iy : cl.iz);
                if (fc.stage_dir > 0 ? im >= mhi : im < mlo) break;   // the next chunk's sample
                float v[8];
                const int ux = cl.ix - bx.lo[0], uy = cl.iy - bx.lo[1], uz = cl.iz - bx.lo[2];
                if (bx.bytes > 0 && ux >= 0 && ux < bx.n[0] - 1 && uy >= 0 && uy < bx.n[1] - 1 && uz >= 0 &&
                    uz < bx.n[2] - 1) {
                    const float *p = stage + ux * so[0] + uy * so[1] + uz * so[2];
                    v[0] = p[0];                  v[1] = p[so[0]];
                    v[2] = p[so[1]];              v[3] = p[so[1] + so[0]];
                    v[4] = p[so[2]];              v[5] = p[so[2] + so[0]];
                    v[6] = p[so[2] + so[1]];      v[7] = p[so[2] + so[1] + so[0]];
                } else {
                    fetch8<0>(src, cl.ix * gst.x + cl.iy * gst.y + cl.iz * gst.z, gst, v);
                }
                if (MASK) mask_channels(v, cl.iz, b.org[2], fc.nz, fc.chmask, fc.vmin);
                DvrSample sm;
                interp_tf(v, cl, false, 1.0f, vmin, inv_range, lutmax, lmax, s_lut, sm);
                over(sm, c0, c1, c2, T);
                ++j;
                jf = __fadd_rn(jf, 1.0f);
                if (T <= thr) done = true;
            }
            if (j >= n) done = true;
            __syncthreads();            // the stage is read before it is refilled
        }
    }
    if (hit && !done && j < n) {        // samples no chunk took (not expected): from global memory
        for (float jf = (float)j; j < n; ++j, jf = __fadd_rn(jf, 1.0f)) {
            const float tj = __fmul_rn(jf, fc.step);
            Cell cl;
            cell_of<true>(__fmaf_rn(tj, d[0], q[0]), __fmaf_rn(tj, d[1], q[1]), __fmaf_rn(tj, d[2], q[2]), mx, my,
                          mz, cl);
            float v[8];
            fetch8<0>(src, cl.ix * gst.x + cl.iy * gst.y + cl.iz * gst.z, gst, v);
            if (MASK) mask_channels(v, cl.iz, b.org[2], fc.nz, fc.chmask, fc.vmin);
            DvrSample sm;
            interp_tf(v, cl, false, 1.0f, vmin, inv_range, lutmax, lmax, s_lut, sm);
            over(sm, c0, c1, c2, T);
            if (T <= thr) { ++j; break; }
        }
    }
    if (inrect) frags[b.frag_off + (long long)ry * rw + rx] = make_float4(c0, c1, c2, T);
    const unsigned int tot = __reduce_add_sync(0xffffffffu, (unsigned int)(hit ? j : 0));
    if (lane == 0 && tot > 0) {
        atomicAdd(&ctr->samples, (unsigned long long)tot);
        if (atomicExch(&b.sampled, 1) == 0) {
            atomicAdd(&ctr->bricks_sampled, 1ull);
            atomicAdd(&ctr->brick_bytes_sampled, (unsigned long long)b.bytes);
        }
    }
}

// ----------------------------------------------------------------------------------------------
// global early termination (occlusion skipping): one pass, each ray walking the bricks
// ----------------------------------------------------------------------------------------------
// Lattice index at which a ray crosses the plane {axis = face}: the binary32 operations of
// box_krange, clamped to +-2^30 before the conversion (far beyond any sampled index, which the
// host keeps below 2^28).  Because a correctly rounded division by step > 0 and the ceiling are
// monotone, a brick's [k0, k1) is the max / min of these indices over its faces, so walking the
// per-axis crossings reproduces every brick's segment exactly.
__device__ __forceinline__ int face_k(float face, float o, float d, float step) {
    const float t = __fdiv_rn(__fdiv_rn(__fsub_rn(face, o), d), step);
    return (int)ceilf(fminf(fmaxf(t, -1073741824.0f), 1073741824.0f));
}

// Sample index at which the ray enters (exit = false) or leaves cell c of an axis (planes
// min(c B, n) and min((c + 1) B, n)); a ray parallel to the axis never crosses.
__device__ __forceinline__ int cell_k(int c, bool exit, float o, float d, float B, float n, float step) {
    if (d == 0.0f) return exit ? 1073741824 : -1073741824;
    const float lo = fminf((float)c * B, n), hi = fminf((float)(c + 1) * B, n);
    const bool upper = (d > 0.0f) == exit;
    return face_k(upper ? hi : lo, o, d, step);
}

// Warps of a global-termination CTA: the CTA is a 32 x kMarchWarps (kMarchWarps x 32) tile of the
// frame, one warp per row (column) of 32 rays.
#ifndef VR_MARCH_WARPS
#define VR_MARCH_WARPS 8
#endif
constexpr int kMarchWarps = VR_MARCH_WARPS;
constexpr int kMarchThreads = 32 * kMarchWarps;

// A march CTA's walk state while its rays sample a segment: one int slot per thread for
// each of the three exits, the three cells, the ray's end, the segment's end, the step bound,
// the sample count, the ray's eye-space offset (two floats) and the pixel's index.  It sits in
// shared memory after the table.
enum MarchSlot { kWkX0, kWkC0 = kWkX0 + 3, kWkK1 = kWkC0 + 3, kWkEnd, kWkGuard, kWkSamp, kWkY0, kWkY1, kWkPix,
                 kWkSlots };
constexpr size_t kMarchStashBytes = (size_t)kWkSlots * kMarchThreads * sizeof(int);

// This thread's first stash slot.  The thread index is read with a volatile move so that the
// address is formed anew at each use instead of held in a register across the sample loop.
__device__ __forceinline__ volatile int *march_stash(float4 *s_lut, int nlut) {
    unsigned tid;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    return reinterpret_cast<volatile int *>(s_lut + 2 * nlut) + tid;
}

// One CTA = a 32x8 (8x32) pixel tile of the frame.  Each ray is clipped to the cube (and the
// render window), then walks the brick grid front to back: its segment in brick b is
// [max(k, enter), min over axes of exit), sampled with the per-brick anchor and stencil of
// the fragment kernel (bit-identical samples), compositing into one running colour and
// transmittance; it stops once the transmittance reaches the threshold after a sample (global
// early termination), so bricks behind opaque pixels cost nothing.  Bricks whose values map
// only to zero opacity are walked through without sampling (their samples add nothing).
// Registers: the sample loop runs with the registers of the fragment kernel's loop plus the
// index clamps; the walk's state rests in shared memory meanwhile (volatile stores and loads
// around each segment, so no register holds it), the origin is rebuilt from the ray's two
// eye-space offsets where a brick or a crossing needs it, and the pixel's index waits in
// shared memory for the final write.
template <int S, int F, bool MASK>
__global__ void __launch_bounds__(kMarchThreads, VR_RAYMARCH_MIN_BLOCKS * 8 / kMarchWarps)
k_raymarch(const FrameConsts fc, const float4 *__restrict__ lut, DrawBrick *__restrict__ bricks,
           const MarchGrid g, const void *__restrict__ pool, float4 *__restrict__ out,
           Counters *__restrict__ ctr) {
    extern __shared__ float4 s_lut[];
    load_table(lut, fc.nlut, s_lut);
    __syncthreads();
    int nsamp = 0;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
    float y0 = 0.0f, y1 = 0.0f, d[3] = {0.0f, 0.0f, 0.0f};
    int K0 = 0, K1 = 0;
    int c[3] = {0, 0, 0}, kx[3] = {0, 0, 0};
    bool ok = false;
    {
        const int tw = fc.lanes_y ? kMarchWarps : kRcLong;
        const int ntx = (fc.cam.W + tw - 1) / tw;
        const int tx = (int)(blockIdx.x % ntx), ty = (int)(blockIdx.x / ntx);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int px = fc.lanes_y ? tx * kMarchWarps + w : tx * kRcLong + lane;
        const int py = fc.lanes_y ? ty * kRcLong + lane : ty * kMarchWarps + w;
        const bool inframe = px < fc.cam.W && py < fc.cam.H;
        march_stash(s_lut, fc.nlut)[kWkPix * kMarchThreads] = inframe ? py * fc.cam.W + px : -1;      // frames hold < 2^31 pixels
        if (inframe) {
            ray_eye(fc.cam, px, py, y0, y1, d);
            float o[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) o[a] = ray_origin(fc.cam, a, y0, y1);
            ok = box_krange(o, d, g.clo, g.chi, fc.step, K0, K1);
            // per axis: the cell owning sample K0 and the index where the ray leaves it
#pragma unroll
            for (int a = 0; a < 3 && ok; ++a) {
                int ca;
                if (d[a] == 0.0f) {
                    // the slab test's own comparisons: the cell with lo <= o < hi
                    ca = clampi((int)floorf(__fmul_rn(o[a], g.invB[a])), 0, g.nb[a] - 1);
                    for (int r = 0; r < g.nb[a]; ++r) {
                        if (ca > 0 && o[a] < fminf((float)ca * g.B[a], g.n[a])) --ca;
                        else if (ca < g.nb[a] - 1 && o[a] >= fminf((float)(ca + 1) * g.B[a], g.n[a])) ++ca;
                        else break;
                    }
                    c[a] = ca;
                    kx[a] = cell_k(ca, true, o[a], d[a], g.B[a], g.n[a], fc.step);
                    ok = K0 < kx[a];
                } else {
                    // an estimate of the cell of sample K0 (any rounding), then settled on the cell
                    // whose [enter, exit) holds K0 by the exact crossings (a step or two at most;
                    // the moves only go one way, so the bound is never reached)
                    const float p = __fmaf_rn(__fmul_rn((float)K0, fc.step), d[a], o[a]);
                    ca = clampi((int)floorf(__fmul_rn(p, g.invB[a])), 0, g.nb[a] - 1);
                    const int step_dir = d[a] > 0.0f ? 1 : -1;
                    int ex = 0, en = 0;
                    bool settled = false;
                    for (int r = 0; r <= g.nb[a] && !settled; ++r) {
                        ex = cell_k(ca, true, o[a], d[a], g.B[a], g.n[a], fc.step);
                        if (ex <= K0 && (unsigned)(ca + step_dir) < (unsigned)g.nb[a]) { ca += step_dir; continue; }
                        en = cell_k(ca, false, o[a], d[a], g.B[a], g.n[a], fc.step);
                        if (en > K0 && (unsigned)(ca - step_dir) < (unsigned)g.nb[a]) { ca -= step_dir; continue; }
                        settled = true;
                    }
                    c[a] = ca;
                    kx[a] = ex;
                    ok = settled && en <= K0 && K0 < ex;
                }
            }
        }
    }
    int k = K0;
    // at most one segment per brick crossed (each step leaves a cell on some axis)
    for (int guard = ok ? g.nb[0] + g.nb[1] + g.nb[2] + 1 : 0; guard > 0 && k < K1; --guard) {
        int kend = min(min(kx[0], kx[1]), min(kx[2], K1));
        const long long bi = ((long long)c[2] * g.nb[1] + c[1]) * g.nb[0] + c[0];
        if (kend > k && !bricks[bi].skip) {
            const DrawBrick &b = bricks[bi];
            const void *src = static_cast<const char *>(pool) + b.data_off * (S == 0 ? 4 : 2);
            const Strides st{b.str[0], b.str[1], b.str[2]};
            const int mx = b.dim[0] - 2, my = b.dim[1] - 2, mz = b.dim[2] - 2;
            const float scale = S == 0 ? 1.0f : ldexpf(1.0f, b.exp2);
            const Atlas atl{gathers(F) ? b.atlas : 0ull, b.alog, b.dim[0], b.dim[1]};
            const float qx = anchor(ray_origin(fc.cam, 0, y0, y1), d[0], b.org_c[0], k, fc.step);
            const float qy = anchor(ray_origin(fc.cam, 1, y0, y1), d[1], b.org_c[1], k, fc.step);
            const float qz = anchor(ray_origin(fc.cam, 2, y0, y1), d[2], b.org_c[2], k, fc.step);
            const int n = kend - k;
            const float vcode = S == 0 ? fc.vmin : ldexpf(fc.vmin, -b.exp2);
            const int org_z = b.org[2];
            volatile int *wk = march_stash(s_lut, fc.nlut);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                wk[(kWkX0 + a) * kMarchThreads] = kx[a];
                wk[(kWkC0 + a) * kMarchThreads] = c[a];
            }
            wk[kWkK1 * kMarchThreads] = K1; wk[kWkEnd * kMarchThreads] = kend; wk[kWkGuard * kMarchThreads] = guard;
            wk[kWkSamp * kMarchThreads] = nsamp;
            wk[kWkY0 * kMarchThreads] = __float_as_int(y0); wk[kWkY1 * kMarchThreads] = __float_as_int(y1);
            const int j = dvr_segment<S, F, true, MASK>(src, st, atl, mx, my, mz, scale, qx, qy, qz, d, n, fc,
                                                        s_lut, org_z, vcode, c0, c1, c2, T);
            wk = march_stash(s_lut, fc.nlut);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                kx[a] = wk[(kWkX0 + a) * kMarchThreads];
                c[a] = wk[(kWkC0 + a) * kMarchThreads];
            }
            K1 = wk[kWkK1 * kMarchThreads]; kend = wk[kWkEnd * kMarchThreads]; guard = wk[kWkGuard * kMarchThreads];
            nsamp = wk[kWkSamp * kMarchThreads] + j;
            y0 = __int_as_float(wk[kWkY0 * kMarchThreads]); y1 = __int_as_float(wk[kWkY1 * kMarchThreads]);
            DrawBrick &bw = bricks[((long long)c[2] * g.nb[1] + c[1]) * g.nb[0] + c[0]];
            if (j > 0 && bw.sampled == 0 && atomicExch(&bw.sampled, 1) == 0) {
                atomicAdd(&ctr->bricks_sampled, 1ull);
                atomicAdd(&ctr->brick_bytes_sampled, (unsigned long long)bw.bytes);
            }
            if (T <= fc.thr) break;               // the whole ray is opaque
        }
        // leave the cells whose exit is here (several at an edge or corner)
        bool out_of_grid = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (kx[a] == kend && kend < K1) {
                c[a] += d[a] > 0.0f ? 1 : -1;
                if ((unsigned)c[a] >= (unsigned)g.nb[a]) out_of_grid = true;
                else kx[a] = cell_k(c[a], true, ray_origin(fc.cam, a, y0, y1), d[a], g.B[a], g.n[a], fc.step);
            }
        }
        if (out_of_grid) break;
        k = kend;
    }
    const int pix = march_stash(s_lut, fc.nlut)[kWkPix * kMarchThreads];
    if (pix >= 0) out[pix] = make_float4(c0, c1, c2, 1.0f - T);
    const unsigned int tot = __reduce_add_sync(0xffffffffu, (unsigned int)nsamp);
    if ((threadIdx.x & 31) == 0 && tot > 0) atomicAdd(&ctr->samples, (unsigned long long)tot);
}

// ----------------------------------------------------------------------------------------------
// compositing: one CTA = one 16x16 screen tile; each pixel blends the fragments of the bricks
// binned to its tile, in the work-list's front-to-back order (Section 2.5)
// ----------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256)
k_composite(const FrameConsts fc, const DrawBrick *__restrict__ dbs, const int *__restrict__ tile_start,
            const int *__restrict__ tile_list, const void *__restrict__ frags, float *__restrict__ out) {
    const int px = blockIdx.x * kTile + (threadIdx.x & 15);
    const int py = blockIdx.y * kTile + (threadIdx.x >> 4);
    if (px >= fc.cam.W || py >= fc.cam.H) return;
    const int t = blockIdx.y * gridDim.x + blockIdx.x;
    const int s0 = tile_start[t], s1 = tile_start[t + 1];
    const long long pix = (long long)py * fc.cam.W + px;
    if (MODE == 0) {
        float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
        for (int e = s0; e < s1; ++e) {
            const DrawBrick &b = dbs[tile_list[e]];
            const int rx = px - b.rect[0], ry = py - b.rect[1];
            if ((unsigned)rx < (unsigned)b.rect[2] && (unsigned)ry < (unsigned)b.rect[3]) {
                const float4 f = static_cast<const float4 *>(frags)[b.frag_off + (long long)ry * b.rect[2] + rx];
                c0 = __fmaf_rn(T, f.x, c0);
                c1 = __fmaf_rn(T, f.y, c1);
                c2 = __fmaf_rn(T, f.z, c2);
                T = __fmul_rn(T, f.w);         // fragment .w holds the segment's transmittance
            }
        }
        reinterpret_cast<float4 *>(out)[pix] = make_float4(c0, c1, c2, fc.sub ? T : 1.0f - T);
    } else {
        float m = -INFINITY;
        for (int e = s0; e < s1; ++e) {
            const DrawBrick &b = dbs[tile_list[e]];
            const int rx = px - b.rect[0], ry = py - b.rect[1];
            if ((unsigned)rx < (unsigned)b.rect[2] && (unsigned)ry < (unsigned)b.rect[3]) {
                const float f = static_cast<const float *>(frags)[b.frag_off + (long long)ry * b.rect[2] + rx];
                m = f > m ? f : m;
            }
        }
        out[pix] = (m == -INFINITY && !fc.sub) ? fc.vmin : m;
    }
}

// Sort-last second stage (Section 2.5): the sub-images of sibling parts, which are consecutive
// slabs of the cube along `axis`, blended per pixel front to back.  A ray crosses the slabs in
// increasing index order when its direction along the axis is positive, in decreasing order
// when negative; with a zero component it meets one slab only, and the others' (0, T = 1) leave
// the blend unchanged whatever the order.  The direction is the ray of that pixel in the
// fragment kernel's own FP32 arithmetic.
__global__ void __launch_bounds__(256)
k_composite_parts(const FrameConsts fc, int axis, int n, const float *__restrict__ subs, int row0, int rows,
                  int final_, float *__restrict__ out) {
    const long long npx = (long long)rows * fc.cam.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npx;
         i += (long long)gridDim.x * blockDim.x) {
        if (fc.mode == 0) {
            const int x = (int)(i % fc.cam.W), y = row0 + (int)(i / fc.cam.W);
            float o[3], d[3];
            ray_for_pixel(fc.cam, x, y, o, d);
            const bool down = d[axis] < 0.0f;
            float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
            for (int j = 0; j < n; ++j) {
                const int k = down ? n - 1 - j : j;
                const float4 f = reinterpret_cast<const float4 *>(subs)[(long long)k * npx + i];
                c0 = __fmaf_rn(T, f.x, c0);
                c1 = __fmaf_rn(T, f.y, c1);
                c2 = __fmaf_rn(T, f.z, c2);
                T = __fmul_rn(T, f.w);
            }
            reinterpret_cast<float4 *>(out)[i] = make_float4(c0, c1, c2, final_ ? 1.0f - T : T);
        } else {
            float m = -INFINITY;
            for (int k = 0; k < n; ++k) {
                const float f = subs[(long long)k * npx + i];
                m = f > m ? f : m;
            }
            out[i] = (m == -INFINITY && final_) ? fc.vmin : m;
        }
    }
}

// ----------------------------------------------------------------------------------------------
// backward pass
// ----------------------------------------------------------------------------------------------
// Composite backward: per pixel, fragments b = 1..B in front-to-back order with premultiplied
// colour C_b and transmittance T_b; C = sum_b P_b C_b, P_b = prod_{b'<b} T_b', output alpha
// A = 1 - prod_b T_b.  Then dL/dC_b = P_b gC and
// dL/dT_b = P_b (gC . Crest_b) - gA P_b Trest_b, with Crest_b / Trest_b the composite of the
// fragments behind b.  Pass 1 (front to back) parks P_b in gfrag.w; pass 2 (back to front)
// accumulates Crest/Trest and writes (dL/dC_b, dL/dT_b).
__global__ void __launch_bounds__(256)
k_composite_backward(const FrameConsts fc, const DrawBrick *__restrict__ dbs,
                     const int *__restrict__ tile_start, const int *__restrict__ tile_list,
                     const float4 *__restrict__ frags, const float4 *__restrict__ gout,
                     float4 *__restrict__ gfrag) {
    const int px = blockIdx.x * kTile + (threadIdx.x & 15);
    const int py = blockIdx.y * kTile + (threadIdx.x >> 4);
    if (px >= fc.cam.W || py >= fc.cam.H) return;
    const int t = blockIdx.y * gridDim.x + blockIdx.x;
    const int s0 = tile_start[t], s1 = tile_start[t + 1];
    const float4 g = gout[(long long)py * fc.cam.W + px];
    float P = 1.0f;
    for (int e = s0; e < s1; ++e) {
        const DrawBrick &b = dbs[tile_list[e]];
        const int rx = px - b.rect[0], ry = py - b.rect[1];
        if ((unsigned)rx < (unsigned)b.rect[2] && (unsigned)ry < (unsigned)b.rect[3]) {
            const long long fi = b.frag_off + (long long)ry * b.rect[2] + rx;
            gfrag[fi].w = P;
            P = __fmul_rn(P, frags[fi].w);
        }
    }
    float r0 = 0.0f, r1 = 0.0f, r2 = 0.0f, Tr = 1.0f;   // composite of the fragments behind
    for (int e = s1 - 1; e >= s0; --e) {
        const DrawBrick &b = dbs[tile_list[e]];
        const int rx = px - b.rect[0], ry = py - b.rect[1];
        if ((unsigned)rx < (unsigned)b.rect[2] && (unsigned)ry < (unsigned)b.rect[3]) {
            const long long fi = b.frag_off + (long long)ry * b.rect[2] + rx;
            const float Pb = gfrag[fi].w;
            const float4 f = frags[fi];
            const float gT = Pb * (g.x * r0 + g.y * r1 + g.z * r2 - g.w * Tr);
            gfrag[fi] = make_float4(Pb * g.x, Pb * g.y, Pb * g.z, gT);
            r0 = fmaf(f.w, r0, f.x);
            r1 = fmaf(f.w, r1, f.y);
            r2 = fmaf(f.w, r2, f.z);
            Tr *= f.w;
        }
    }
}

// A ray's cell accumulator after one step along axis SH (up: +1): the corners of the face both
// cells share move to their place in the new cell, the new far face starts empty.
template <int SH>
__device__ __forceinline__ void shift_face(float acc[8], bool up) {
    float nacc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const bool hi = (c >> SH) & 1;
        nacc[c] = up ? (hi ? 0.0f : acc[c ^ (1 << SH)]) : (hi ? acc[c ^ (1 << SH)] : 0.0f);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = nacc[c];
}

// Adds a ray's accumulated voxel gradients of cell (cx, cy, cz) (corner c = x + 2y + 4z) for
// the corners in `mask` to the cube's gradient (ghost copies map back to their source voxel).
__device__ __forceinline__ void flush_voxel_grads(float *__restrict__ gvox, const float acc[8], unsigned mask,
                                                  int cx, int cy, int cz, const DrawBrick &b,
                                                  const FrameConsts &fc) {
    const int x0 = clampi(b.org[0] + cx, 0, fc.nx - 1), x1 = clampi(b.org[0] + cx + 1, 0, fc.nx - 1);
    const int y0 = clampi(b.org[1] + cy, 0, fc.ny - 1), y1 = clampi(b.org[1] + cy + 1, 0, fc.ny - 1);
    const int z0 = clampi(b.org[2] + cz, 0, fc.nz - 1), z1 = clampi(b.org[2] + cz + 1, 0, fc.nz - 1);
    // corner (0,0,0)'s address once, the other corners as 32-bit steps from it (a step along an
    // axis is one voxel's stride, or 0 where the cube's border clamps both corners together)
    float *p = gvox + ((long long)z0 * fc.ny + y0) * fc.nx + x0;
    const int dx = x1 - x0, dy = (y1 - y0) * fc.nx;
    const long long dz = (long long)(z1 - z0) * fc.nx * fc.ny;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (((mask >> c) & 1u) && acc[c] != 0.0f)
            atomicAdd(p + ((c & 1) ? dx : 0) + ((c & 2) ? dy : 0) + ((c & 4) ? dz : 0), acc[c]);
}

// Adjoint ray cast (FP32 bricks).  Each (brick, pixel) segment is replayed front to back with
// the forward's arithmetic; from the stored segment colour C_b and transmittance T_b the
// gradient of every sample follows without per-sample storage:
//   dL/dc_j = gC T_{j-1} a_j
//   dL/da_j = T_{j-1} [ gC.c_j - (gC.(C_b - C_{<=j}) + gT T_b) / T_j ]   (T_j = T_{j-1}(1-a_j))
//   last composited sample: dL/da_j = T_{j-1} [ gC.c_j - gT ]
// Table gradients accumulate per CTA in a partial row in L2 (two float4 atomics per sample; eight
// float atomics per sample into shared-memory copies were 13 % slower per batch, their retries of
// contended adds and the copy-out included).
// Voxel gradients accumulate per ray for the 8 corners of its current cell and are added to the
// cube's voxels when the ray leaves the cell (ghost copies map back to their source voxel); a
// step into an adjacent cell keeps the shared face's 4 sums (before: 8 atomics per sample).
// Bounded to 4 CTAs per SM (64 registers, a few spilled; 80 unbounded give 3 CTAs, 8 % slower).
// ATLAS: the replay reads the stencils from the bricks' slice atlases (the forward's texels)
// instead of the linear copy.
template <bool ATLAS>
__global__ void __launch_bounds__(256, VR_ADJ_MIN_BLOCKS)
k_adjoint(const FrameConsts fc, const float4 *__restrict__ lut, const DrawBrick *__restrict__ dbs,
          const TileItem *__restrict__ items, const float *__restrict__ pool,
          const float4 *__restrict__ frags, const float4 *__restrict__ gfrag,
          float *__restrict__ glut_partial, float *__restrict__ gvox) {
    extern __shared__ float4 s_lut[];
    load_table(lut, fc.nlut, s_lut);
    __syncthreads();
    const TileItem it = items[blockIdx.x];
    const DrawBrick &b = dbs[it.db];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's table-gradient partial: one float4 (the 4 channels) per entry, zeroed before the
    // launch; each sample adds its two entries' channels with one vector atomic each (in L2)
    float4 *g_row = reinterpret_cast<float4 *>(glut_partial) + (long long)blockIdx.x * fc.nlut;
    // a warp's 32 rays are adjacent pixels along the image axis the brick layout follows
    int rx, ry;
    thread_pixel(fc.lanes_y, it, warp, lane, rx, ry);
    if (rx < b.rect[2] && ry < b.rect[3]) {
        const long long fi = b.frag_off + (long long)ry * b.rect[2] + rx;
        const float4 gf = gfrag[fi];
        float o[3], d[3];
        ray_for_pixel(fc.cam, b.rect[0] + rx, b.rect[1] + ry, o, d);
        int k0 = 0, k1 = 0;
        if ((gf.x != 0.0f || gf.y != 0.0f || gf.z != 0.0f || gf.w != 0.0f) &&
            box_krange(o, d, b.lo, b.hi, fc.step, k0, k1)) {
            const float4 fr = frags[fi];
            const float *src = pool + b.data_off;
            const Strides st{b.str[0], b.str[1], b.str[2]};
            const int mx = b.dim[0] - 2, my = b.dim[1] - 2, mz = b.dim[2] - 2;
            const float qx = anchor(o[0], d[0], b.org_c[0], k0, fc.step);
            const float qy = anchor(o[1], d[1], b.org_c[1], k0, fc.step);
            const float qz = anchor(o[2], d[2], b.org_c[2], k0, fc.step);
            const int n = k1 - k0;
            const float dxdv = __fmul_rn(fc.lutmax, fc.inv_range);
            float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, T = 1.0f;
            // voxel gradients of the ray's current cell, added to the cube when the ray leaves it
            float acc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            int ccx = -4, ccy = -4, ccz = -4;
            const Atlas atl{ATLAS ? b.atlas : 0ull, b.alog, b.dim[0], b.dim[1]};
            for (int j = 0; j < n; ++j) {
                const float tj = __fmul_rn((float)j, fc.step);
                DvrSample sm;
                dvr_sample<0>(src, st, mx, my, mz, 1.0f, __fmaf_rn(tj, d[0], qx),
                              __fmaf_rn(tj, d[1], qy), __fmaf_rn(tj, d[2], qz), fc.vmin,
                              fc.inv_range, fc.lutmax, fc.nlut - 2, s_lut, fc.chmask, b.org[2],
                              fc.nz, fc.vmin, sm, ATLAS ? &atl : nullptr);
                const float Tb = T;
                over(sm, c0, c1, c2, T);
                const bool last = (T <= fc.thr) || (j == n - 1);
                const float gcdot = gf.x * sm.r + gf.y * sm.g + gf.z * sm.b;
                float ga;
                if (last) {
                    ga = Tb * (gcdot - gf.w);
                } else {
                    const float sdot = gf.x * (fr.x - c0) + gf.y * (fr.y - c1) + gf.z * (fr.z - c2);
                    ga = Tb * (gcdot - (sdot + gf.w * fr.w) / T);
                }
                const float wa = Tb * sm.a;
                const float gr = gf.x * wa, gg = gf.y * wa, gb = gf.z * wa;
                const float w1 = sm.lf, w0 = 1.0f - sm.lf;
                atomicAdd(g_row + sm.li, make_float4(w0 * gr, w0 * gg, w0 * gb, w0 * ga));
                if (sm.li + 1 < fc.nlut)      // the last entry (u >= 1) has weight 1 and no next entry
                    atomicAdd(g_row + sm.li + 1, make_float4(w1 * gr, w1 * gg, w1 * gb, w1 * ga));
                if (gvox != nullptr && sm.u > 0.0f && sm.u < 1.0f) {
                    const float gx = gr * sm.D.x + gg * sm.D.y + gb * sm.D.z + ga * sm.D.w;
                    const float gv = gx * dxdv;
                    if (gv != 0.0f) {
                        const int ix = sm.ix, iy = sm.iy, iz = sm.iz;
                        if (ix != ccx || iy != ccy || iz != ccz) {
                            const int ddx = ix - ccx, ddy = iy - ccy, ddz = iz - ccz;
                            const int ax = (ddx != 0) + (ddy != 0) + (ddz != 0);
                            if (ax == 1 && ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1 &&
                                ddz >= -1 && ddz <= 1) {
                                // one step along one axis: the face both cells share keeps accumulating
                                const int sh = ddx != 0 ? 0 : (ddy != 0 ? 1 : 2);
                                const int up = (ddx + ddy + ddz) > 0;
                                const unsigned lowf = sh == 0 ? 0x55u : (sh == 1 ? 0x33u : 0x0Fu);
                                flush_voxel_grads(gvox, acc, up ? lowf : (~lowf & 0xffu), ccx, ccy, ccz, b, fc);
                                if (sh == 0) shift_face<0>(acc, up);
                                else if (sh == 1) shift_face<1>(acc, up);
                                else shift_face<2>(acc, up);
                            } else {
                                flush_voxel_grads(gvox, acc, 0xffu, ccx, ccy, ccz, b, fc);
#pragma unroll
                                for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
                            }
                            ccx = ix; ccy = iy; ccz = iz;
                        }
                        const int gz0 = clampi(b.org[2] + iz, 0, fc.nz - 1), gz1 = clampi(b.org[2] + iz + 1, 0, fc.nz - 1);
                        const float ux = sm.fx, uy = sm.fy;
                        const float vx = 1.0f - ux, vy = 1.0f - uy;
                        const float uz = (fc.chmask && !fc.chmask[gz1]) ? 0.0f : sm.fz;
                        const float vz = (fc.chmask && !fc.chmask[gz0]) ? 0.0f : 1.0f - sm.fz;
                        // trilinear weights of the 8 corners, factored by z, then y
                        const float wz0 = gv * vz, wz1 = gv * uz;
                        const float g00 = wz0 * vy, g10 = wz0 * uy, g01 = wz1 * vy, g11 = wz1 * uy;
                        acc[0] = __fmaf_rn(g00, vx, acc[0]); acc[1] = __fmaf_rn(g00, ux, acc[1]);
                        acc[2] = __fmaf_rn(g10, vx, acc[2]); acc[3] = __fmaf_rn(g10, ux, acc[3]);
                        acc[4] = __fmaf_rn(g01, vx, acc[4]); acc[5] = __fmaf_rn(g01, ux, acc[5]);
                        acc[6] = __fmaf_rn(g11, vx, acc[6]); acc[7] = __fmaf_rn(g11, ux, acc[7]);
                    }
                }
                if (T <= fc.thr) break;
            }
            if (gvox != nullptr && ccx != -4) flush_voxel_grads(gvox, acc, 0xffu, ccx, ccy, ccz, b, fc);
        }
    }
}

// Final reduction of the per-CTA table-gradient partials, in FP64 and in two stages so that
// every entry's sum is spread over many threads yet formed in a fixed order: chunk y sums the
// partials of parts [y q, (y + 1) q) in part order, then the chunk sums are added in chunk order.
__global__ void k_lut_grad_chunks(const float *__restrict__ partial, int nparts, int n, double *__restrict__ chunks) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int q = (nparts + (int)gridDim.y - 1) / (int)gridDim.y;
    const int p0 = (int)blockIdx.y * q, p1 = min(nparts, p0 + q);
    double a = 0.0;
    for (int p = p0; p < p1; ++p) a += (double)partial[(long long)p * n + i];
    chunks[(long long)blockIdx.y * n + i] = a;
}

__global__ void k_lut_grad_reduce(const double *__restrict__ chunks, int nchunks, int n, float *__restrict__ glut) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int y = 0; y < nchunks; ++y) acc += chunks[(long long)y * n + i];
    glut[i] = (float)acc;
}

// Several views' table gradients: each view's chunk sums are added to one FP64 accumulator
// (zeroed by the first view), which is rounded to FP32 once, after the last view.
__global__ void k_lut_grad_accumulate(const double *__restrict__ chunks, int nchunks, int n,
                                      double *__restrict__ acc, int first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = first ? 0.0 : acc[i];
    for (int y = 0; y < nchunks; ++y) a += chunks[(long long)y * n + i];
    acc[i] = a;
}

__global__ void k_lut_grad_store(const double *__restrict__ acc, int n, float *__restrict__ glut) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) glut[i] = (float)acc[i];
}

// Function attributes (the dynamic shared-memory limit, the carveout) are set per device: a
// kernel's attributes on one GPU say nothing about another GPU of the same process.  Each
// launcher remembers what it set in one slot per device ordinal (devices beyond kAttrDevices
// are set on every launch).  Frames of the serving loop may launch from several host threads:
// the slots are atomics, and setting an attribute twice is harmless.
constexpr int kAttrDevices = 64;
struct DeviceAttrs {
    std::atomic<int> smem[kAttrDevices];     // dynamic shared-memory limit set (bytes), 0: not yet
    std::atomic<int> carve[kAttrDevices];    // carveout percentage set, -1: not yet
    DeviceAttrs() {
        for (int i = 0; i < kAttrDevices; ++i) { smem[i].store(0); carve[i].store(-1); }
    }
};

int current_device() {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}

// Raises the kernel's dynamic shared-memory limit to `bytes` on the current device (once).
cudaError_t ensure_smem_limit(const void *kernel, int bytes, DeviceAttrs &da) {
    const int dev = current_device();
    const bool cached = dev >= 0 && dev < kAttrDevices;
    if (cached && da.smem[dev].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && cached) da.smem[dev].store(bytes, std::memory_order_release);
    return e;
}

// The unified L1 / shared memory of an SM serves the texture gathers as cache: ask for just the
// shared memory (the table) of the CTAs of `warps` warps the register file admits, leaving the
// rest to L1 (measured on HIPASS-scale frames at 5 CTAs: 25 % carveout 3.65 ms, the driver's
// default 3.75, 50 % 3.98).  Registers are allocated per warp in units of 256, 64 K per SM, at
// most 64 warps and 32 CTAs.  The kernel's current preference on this device is remembered in
// `da`.
cudaError_t set_carveout(const void *kernel, size_t smem_per_cta, DeviceAttrs &da, int warps = 8) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int ctas = std::max(1, std::min(32, std::min(64, 65536 / std::max(per_warp, 256)) / warps));
    const double need = ctas * (double)(smem_per_cta + 1024) / (228.0 * 1024.0);
    const int pct = std::min(100, std::max(0, (int)std::ceil(100.0 * need)));
    const int dev = current_device();
    const bool cached = dev >= 0 && dev < kAttrDevices;
    if (cached && da.carve[dev].load(std::memory_order_relaxed) == pct) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    if (e == cudaSuccess && cached) da.carve[dev].store(pct, std::memory_order_relaxed);
    return e;
}

template <int S, int MODE, int F, bool MASK>
cudaError_t launch_rc(const FrameConsts &fc, const float4 *lut, const DrawBrick *db, const TileItem *items,
                      int nitems, const void *pool, void *frags, Counters *ctr, cudaStream_t s) {
    static DeviceAttrs da;
    const size_t smem = MODE == 0 ? 2 * sizeof(float4) * (size_t)fc.nlut : 0;
    const void *kern = reinterpret_cast<const void *>(k_raycast<S, MODE, F, MASK>);
    cudaError_t e = ensure_smem_limit(kern, (int)(2 * sizeof(float4) * kMaxLut), da);
    if (e != cudaSuccess) return e;
    if (MODE == 0) {
        e = set_carveout(kern, smem, da);
        if (e != cudaSuccess) return e;
    }
    k_raycast<S, MODE, F, MASK><<<nitems, 256, smem, s>>>(fc, lut, const_cast<DrawBrick *>(db), items, pool, frags, ctr);
    return cudaGetLastError();
}

template <bool MASK>
cudaError_t launch_staged(const FrameConsts &fc, const float4 *lut, const DrawBrick *db, const TileItem *items,
                          int nitems, const void *pool, void *frags, Counters *ctr, cudaStream_t s) {
    static DeviceAttrs da;
    const size_t smem = 2 * sizeof(float4) * (size_t)fc.nlut + 2 * sizeof(float) * (size_t)kStageFloats;
    const void *kern = reinterpret_cast<const void *>(k_raycast_staged<MASK>);
    cudaError_t e = ensure_smem_limit(kern, (int)(2 * sizeof(float4) * kMaxLut + 2 * sizeof(float) * kStageFloats), da);
    if (e != cudaSuccess) return e;
    k_raycast_staged<MASK><<<nitems, 256, smem, s>>>(fc, lut, const_cast<DrawBrick *>(db), items,
                                                     static_cast<const float *>(pool), static_cast<float4 *>(frags), ctr);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_rc_s(const FrameConsts &fc, const float4 *lut, const DrawBrick *db, const TileItem *items,
                        int nitems, const void *pool, void *frags, Counters *ctr, cudaStream_t s) {
    if (S == 0 && fc.fetch == 4 && fc.mode == 0)
        return fc.chmask ? launch_staged<true>(fc, lut, db, items, nitems, pool, frags, ctr, s)
                         : launch_staged<false>(fc, lut, db, items, nitems, pool, frags, ctr, s);
#define VR_RC(MODE, F, MASK) launch_rc<S, MODE, F, MASK>(fc, lut, db, items, nitems, pool, frags, ctr, s)
    if constexpr (S != 0) {           // pair atlases: 16-bit bricks only
        if (fc.fetch == 5) {
            if (fc.chmask) return fc.mode != 0 ? VR_RC(1, 5, true) : VR_RC(0, 5, true);
            return fc.mode != 0 ? VR_RC(1, 5, false) : VR_RC(0, 5, false);
        }
    }
    const bool atlas = fc.fetch == 2;
    if (fc.chmask) {     // masked frames: no stencil cache (same values, fewer instantiations)
        if (fc.mode != 0) return atlas ? VR_RC(1, 2, true) : VR_RC(1, 0, true);
        return atlas ? VR_RC(0, 2, true) : VR_RC(0, 0, true);
    }
    if (fc.mode != 0) return atlas ? VR_RC(1, 2, false) : VR_RC(1, 0, false);
    if (atlas) return VR_RC(0, 2, false);
    if (fc.fetch == 1) return VR_RC(0, 1, false);
    return VR_RC(0, 0, false);
#undef VR_RC
}

}  // namespace

cudaError_t launch_raycast(const FrameConsts &fc, const float4 *lut, const DrawBrick *db,
                           const TileItem *items, int nitems, const void *pool, void *frags,
                           Counters *ctr, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (fc.storage == 0) return launch_rc_s<0>(fc, lut, db, items, nitems, pool, frags, ctr, s);
    if (fc.storage == 1) return launch_rc_s<1>(fc, lut, db, items, nitems, pool, frags, ctr, s);
    return launch_rc_s<2>(fc, lut, db, items, nitems, pool, frags, ctr, s);
}

template <int S, int F, bool MASK>
cudaError_t launch_march(const FrameConsts &fc, const float4 *lut, DrawBrick *bricks, const MarchGrid &g,
                         const void *pool, float4 *out, Counters *ctr, cudaStream_t s) {
    static DeviceAttrs da;
    const void *kern = reinterpret_cast<const void *>(k_raymarch<S, F, MASK>);
    cudaError_t e = ensure_smem_limit(kern, (int)(2 * sizeof(float4) * kMaxLut + kMarchStashBytes), da);
    const size_t smem = 2 * sizeof(float4) * (size_t)fc.nlut + kMarchStashBytes;
    if (e == cudaSuccess) e = set_carveout(kern, smem, da, kMarchWarps);
    if (e != cudaSuccess) return e;
    const int tw = fc.lanes_y ? kMarchWarps : kRcLong, th = fc.lanes_y ? kRcLong : kMarchWarps;
    const long long ntiles = (long long)((fc.cam.W + tw - 1) / tw) * ((fc.cam.H + th - 1) / th);
    k_raymarch<S, F, MASK><<<(unsigned)ntiles, kMarchThreads, smem, s>>>(fc, lut, bricks, g, pool, out, ctr);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_march_s(const FrameConsts &fc, const float4 *lut, DrawBrick *bricks, const MarchGrid &g,
                           const void *pool, float4 *out, Counters *ctr, cudaStream_t s) {
    if constexpr (S != 0) {           // pair atlases: 16-bit bricks only
        if (fc.fetch == 5)
            return fc.chmask ? launch_march<S, 5, true>(fc, lut, bricks, g, pool, out, ctr, s)
                             : launch_march<S, 5, false>(fc, lut, bricks, g, pool, out, ctr, s);
    }
    const bool atlas = fc.fetch == 2;
    if (fc.chmask)
        return atlas ? launch_march<S, 2, true>(fc, lut, bricks, g, pool, out, ctr, s)
                     : launch_march<S, 0, true>(fc, lut, bricks, g, pool, out, ctr, s);
    return atlas ? launch_march<S, 2, false>(fc, lut, bricks, g, pool, out, ctr, s)
                 : launch_march<S, 0, false>(fc, lut, bricks, g, pool, out, ctr, s);
}

cudaError_t launch_raymarch(const FrameConsts &fc, const float4 *lut, DrawBrick *bricks, const MarchGrid &g,
                            const void *pool, float4 *out, Counters *ctr, cudaStream_t s) {
    if (fc.storage == 0) return launch_march_s<0>(fc, lut, bricks, g, pool, out, ctr, s);
    if (fc.storage == 1) return launch_march_s<1>(fc, lut, bricks, g, pool, out, ctr, s);
    return launch_march_s<2>(fc, lut, bricks, g, pool, out, ctr, s);
}

cudaError_t launch_composite(const FrameConsts &fc, const DrawBrick *db, const int *tile_start,
                             const int *tile_list, const void *frags, float *out, cudaStream_t s) {
    dim3 grid((fc.cam.W + kTile - 1) / kTile, (fc.cam.H + kTile - 1) / kTile);
    if (fc.mode == 0)
        k_composite<0><<<grid, 256, 0, s>>>(fc, db, tile_start, tile_list, frags, out);
    else
        k_composite<1><<<grid, 256, 0, s>>>(fc, db, tile_start, tile_list, frags, out);
    return cudaGetLastError();
}

cudaError_t launch_composite_parts(const FrameConsts &fc, int axis, int n, const float *subs, int row0, int rows,
                                   int final_, float *out, cudaStream_t s) {
    const long long npx = (long long)rows * fc.cam.W;
    if (npx <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((npx + 255) / 256, 152 * 8);
    k_composite_parts<<<grid, 256, 0, s>>>(fc, axis, n, subs, row0, rows, final_, out);
    return cudaGetLastError();
}

cudaError_t launch_composite_backward(const FrameConsts &fc, const DrawBrick *db,
                                      const int *tile_start, const int *tile_list,
                                      const float4 *frags, const float4 *gout, float4 *gfrag,
                                      cudaStream_t s) {
    dim3 grid((fc.cam.W + kTile - 1) / kTile, (fc.cam.H + kTile - 1) / kTile);
    k_composite_backward<<<grid, 256, 0, s>>>(fc, db, tile_start, tile_list, frags, gout, gfrag);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const FrameConsts &fc, const float4 *lut, const DrawBrick *db,
                           const TileItem *items, int nitems, const float *pool,
                           const float4 *frags, const float4 *gfrag, float *glut_partial,
                           float *gvox, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    static DeviceAttrs da_lin, da_atl;
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void *>(k_adjoint<false>), (int)(32 * kMaxLut), da_lin);
    if (e == cudaSuccess)
        e = ensure_smem_limit(reinterpret_cast<const void *>(k_adjoint<true>), (int)(32 * kMaxLut), da_atl);
    if (e != cudaSuccess) return e;
    const size_t smem = 32 * (size_t)fc.nlut;      // table + differences
    e = cudaMemsetAsync(glut_partial, 0, sizeof(float) * 4 * (size_t)fc.nlut * nitems, s);
    if (e != cudaSuccess) return e;
    if (fc.fetch == 2)
        k_adjoint<true><<<nitems, 256, smem, s>>>(fc, lut, db, items, pool, frags, gfrag, glut_partial, gvox);
    else
        k_adjoint<false><<<nitems, 256, smem, s>>>(fc, lut, db, items, pool, frags, gfrag, glut_partial, gvox);
    return cudaGetLastError();
}

static cudaError_t launch_lut_grad_chunks(const float *partial, int nparts, int n, double *chunks, cudaStream_t s) {
    dim3 grid((n + 255) / 256, kLutGradChunks);
    k_lut_grad_chunks<<<grid, 256, 0, s>>>(partial, nparts, n, chunks);
    return cudaGetLastError();
}

cudaError_t launch_lut_grad_reduce(const float *partial, int nparts, int nlut, double *chunks, float *glut,
                                   cudaStream_t s) {
    const int n = 4 * nlut;
    cudaError_t e = launch_lut_grad_chunks(partial, nparts, n, chunks, s);
    if (e != cudaSuccess) return e;
    k_lut_grad_reduce<<<(n + 255) / 256, 256, 0, s>>>(chunks, kLutGradChunks, n, glut);
    return cudaGetLastError();
}

cudaError_t launch_lut_grad_accumulate(const float *partial, int nparts, int nlut, double *chunks, double *acc,
                                       bool first, cudaStream_t s) {
    const int n = 4 * nlut;
    cudaError_t e = launch_lut_grad_chunks(partial, nparts, n, chunks, s);
    if (e != cudaSuccess) return e;
    k_lut_grad_accumulate<<<(n + 255) / 256, 256, 0, s>>>(chunks, kLutGradChunks, n, acc, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_lut_grad_store(const double *acc, int nlut, float *glut, cudaStream_t s) {
    const int n = 4 * nlut;
    k_lut_grad_store<<<(n + 255) / 256, 256, 0, s>>>(acc, n, glut);
    return cudaGetLastError();
}

}  // namespace vr
