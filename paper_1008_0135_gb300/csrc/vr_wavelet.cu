// vr_wavelet.cu -- lossy wavelet compression of a cube kept in GPU memory (Section 6: wavelet
// compression of the cube portions stored in GPU memory, with fast decompression and random
// access, to store and render larger cubes).
//
// The cube is cut into 8x8x8 blocks on a global grid (border blocks padded by repeating the
// edge voxels).  Each block is transformed by three levels of the 3D Haar average/difference
// transform, s = (a + b)/2, d = (a - b)/2 along x, then y, then z, each level on the
// previous level's averages; the 511 detail coefficients are quantised to int8 with one
// power-of-two step per subband and the average is kept in FP32.  A block is one fixed-size
// record, so any block decodes on its own (random access at block granularity).  Every
// operation is an explicit IEEE binary32 operation in a fixed order, so the codes and the
// decoded values are exact functions of the input.
//
// Record (kWaveletRecordBytes = 544 bytes):
//   [0, 512)   int8 q[x + 8 y + 64 z] in the block's pyramid layout (entry 0 unused, 0)
//   [512, 516) FP32 average of the block (the level-3 approximation)
//   [516, 537) int8 e[7 (L - 1) + (bx + 2 by + 4 bz) - 1], the step 2^e of subband (bx, by, bz)
//              of level L; -128: the subband is all zero
//   [537, 544) zero
// Coefficient (x, y, z) belongs to level L (n = 8 >> (L - 1), h = n / 2) when it lies in
// [0, n)^3 but not in [0, h)^3, to subband bx = (x >= h), by = (y >= h), bz = (z >= h).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "vr_internal.cuh"

namespace vr {
namespace {

constexpr int kWarpsPerCta = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// level and subband slot (7 (L - 1) + sb - 1) of pyramid position p = x + 8 y + 64 z; -1: average
__device__ __forceinline__ int subband_of(int p) {
    const int x = p & 7, y = (p >> 3) & 7, z = p >> 6;
    const int m = max(x, max(y, z));
    if (m == 0) return -1;
    const int L = m >= 4 ? 1 : (m >= 2 ? 2 : 3);
    const int h = 4 >> (L - 1);
    const int sb = (x >= h ? 1 : 0) + (y >= h ? 2 : 0) + (z >= h ? 4 : 0);
    return 7 * (L - 1) + sb - 1;
}

// One level of the forward transform on the sub-cube [0, n)^3 of a (8x8x8, x fastest), using
// b as scratch; one warp.  Along x, then y, then z.
__device__ void haar_forward_level(float *a, float *b, int n, int lane) {
    const int h = n >> 1;
    for (int axis = 0; axis < 3; ++axis) {
        const int st = axis == 0 ? 1 : (axis == 1 ? 8 : 64);
        for (int t = lane; t < n * n * h; t += 32) {
            // t = i + h (u + n v): pair i of the line at (u, v) across the other two axes
            const int i = t % h, r = t / h, u = r % n, v = r / n;
            int base;
            if (axis == 0) base = 8 * u + 64 * v;
            else if (axis == 1) base = u + 64 * v;
            else base = u + 8 * v;
            const float x0 = a[base + (2 * i) * st], x1 = a[base + (2 * i + 1) * st];
            b[base + i * st] = __fmul_rn(__fadd_rn(x0, x1), 0.5f);
            b[base + (h + i) * st] = __fmul_rn(__fsub_rn(x0, x1), 0.5f);
        }
        __syncwarp();
        for (int t = lane; t < n * n * n; t += 32) {
            const int x = t % n, y = (t / n) % n, z = t / (n * n);
            const int p = x + 8 * y + 64 * z;
            a[p] = b[p];
        }
        __syncwarp();
    }
}

// 2^k as a float for k in [-126, 127] (built from its bits: exact).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Encoder: one warp per block.
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_wavelet_encode(const float *__restrict__ cube, int nx, int ny, int nz, int bnx, int bny, long long nblocks,
                 unsigned char *__restrict__ store) {
    __shared__ float s_a[kWarpsPerCta][512];
    __shared__ float s_b[kWarpsPerCta][512];
    __shared__ unsigned int s_max[kWarpsPerCta][21];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long blk = (long long)blockIdx.x * kWarpsPerCta + w;
    if (blk >= nblocks) return;                      // warp-uniform; no block-wide barrier below
    float *a = s_a[w], *b = s_b[w];
    const int bx = (int)(blk % bnx), by = (int)((blk / bnx) % bny), bz = (int)(blk / ((long long)bnx * bny));
    for (int p = lane; p < 512; p += 32) {
        const int x = clampi(8 * bx + (p & 7), 0, nx - 1), y = clampi(8 * by + ((p >> 3) & 7), 0, ny - 1);
        const int z = clampi(8 * bz + (p >> 6), 0, nz - 1);
        a[p] = cube[((long long)z * ny + y) * nx + x];
    }
    if (lane < 21) s_max[w][lane] = 0u;
    __syncwarp();
    haar_forward_level(a, b, 8, lane);
    haar_forward_level(a, b, 4, lane);
    haar_forward_level(a, b, 2, lane);
    for (int p = lane; p < 512; p += 32) {
        const int sb = subband_of(p);
        if (sb >= 0) atomicMax(&s_max[w][sb], __float_as_uint(fabsf(a[p])));
    }
    __syncwarp();
    unsigned char *rec = store + blk * kWaveletRecordBytes;
    __shared__ int s_e[kWarpsPerCta][21];
    if (lane < 21) {
        const float m = __uint_as_float(s_max[w][lane]);
        int e = -128;
        if (m > 0.0f) {
            int k;
            frexpf(m, &k);                           // m = f 2^k, 1/2 <= f < 1
            e = k - 7;
            if (e >= -126 && m > __fmul_rn(127.0f, pow2f(e))) e += 1;
            e = clampi(e, -126, 120);
        }
        s_e[w][lane] = e;
        rec[516 + lane] = (unsigned char)(signed char)e;
    }
    if (lane < 7) rec[537 + lane] = 0;
    __syncwarp();
    // codes, 4 per 32-bit word
    for (int q4 = lane; q4 < 128; q4 += 32) {
        unsigned int word = 0;
        for (int j = 0; j < 4; ++j) {
            const int p = 4 * q4 + j;
            const int sb = subband_of(p);
            int q = 0;
            if (sb >= 0) {
                const int e = s_e[w][sb];
                if (e != -128) q = clampi((int)rintf(__fmul_rn(a[p], pow2f(-e))), -127, 127);
            }
            word |= (unsigned int)(q & 0xff) << (8 * j);
        }
        reinterpret_cast<unsigned int *>(rec)[q4] = word;
    }
    if (lane == 0) *reinterpret_cast<float *>(rec + 512) = a[0];
}

// Inverse of one level for one 2x2x2 group: c[a + 2b + 4c] holds the coarser average (c[0]) and
// the 7 details of subbands (a, b, c); the separable inverse pairs along z, then y, then x
// touch only these 8 values, so out[x + 2y + 4z] here is bit-identical to the whole-level
// passes (same pairs, same binary32 operations, same order).
__device__ __forceinline__ void inv_group(const float c[8], float out[8]) {
    float t[8], u[8];
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) {              // along z
        t[ab] = __fadd_rn(c[ab], c[ab + 4]);
        t[ab + 4] = __fsub_rn(c[ab], c[ab + 4]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {                 // along y: r = a + 4z -> index a + 4z (+ 2)
        const int i0 = (r & 1) + 4 * (r >> 1);
        u[i0] = __fadd_rn(t[i0], t[i0 + 2]);
        u[i0 + 2] = __fsub_rn(t[i0], t[i0 + 2]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {                 // along x: r = y + 2z -> index 2y + 4z (+ 1)
        const int i0 = 2 * r;
        out[i0] = __fadd_rn(u[i0], u[i0 + 1]);
        out[i0 + 1] = __fsub_rn(u[i0], u[i0 + 1]);
    }
}

// Dequantised coefficient of pyramid position p (detail of subband slot sb) from shared codes.
__device__ __forceinline__ float coef(const signed char *q, const float *step, int p, int slot) {
    return __fmul_rn((float)q[p], step[slot]);
}

// One level for group (i, j, k) of half-size h = 4 >> (L - 1): the average comes from `avg`, the
// details from the pyramid positions (i + a h, j + b h, k + c h).
__device__ __forceinline__ void level_group(const signed char *q, const float *step, int L, int i, int j, int k,
                                            float avg, float out[8]) {
    const int h = 4 >> (L - 1);
    float c[8];
    c[0] = avg;
#pragma unroll
    for (int sb = 1; sb < 8; ++sb) {
        const int p = (i + (sb & 1) * h) + 8 * (j + ((sb >> 1) & 1) * h) + 64 * (k + (sb >> 2) * h);
        c[sb] = coef(q, step, p, 7 * (L - 1) + sb - 1);
    }
    inv_group(c, out);
}

// Decoder into one brick's stored region: elements (x, y, z) of a dx*dy*dz x-contiguous FP32
// array holding global voxel clamp(org + (x, y, z)).  One warp per cube block that the
// region's clamped coordinates touch: levels 3 and 2 on a few lanes, level 1 as 64 independent
// 2x2x2 groups (two per lane), the block's 512 voxels in shared memory, then written to every
// element that maps to them.
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_wavelet_decode(const unsigned char *__restrict__ store, int nx, int ny, int nz, int bnx, int bny,
                 int ox, int oy, int oz, int dx, int dy, int dz, int b0x, int b0y, int b0z, int nbx, int nby,
                 long long nbl, float *__restrict__ dst) {
    __shared__ __align__(16) signed char s_q[kWarpsPerCta][512];
    __shared__ float s_step[kWarpsPerCta][21];
    __shared__ float s_l3[kWarpsPerCta][8];
    __shared__ float s_l2[kWarpsPerCta][64];
    __shared__ float s_v[kWarpsPerCta][512];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * kWarpsPerCta + w;
    if (t >= nbl) return;                             // warp-uniform
    const int cbx = b0x + (int)(t % nbx), cby = b0y + (int)((t / nbx) % nby), cbz = b0z + (int)(t / ((long long)nbx * nby));
    const unsigned char *rec = store + (((long long)cbz * bny + cby) * bnx + cbx) * kWaveletRecordBytes;
    reinterpret_cast<uint4 *>(s_q[w])[lane] = reinterpret_cast<const uint4 *>(rec)[lane];
    if (lane < 21) {
        const int e = (int)(signed char)rec[516 + lane];
        s_step[w][lane] = e == -128 ? 0.0f : pow2f(e);
    }
    const float avg = *reinterpret_cast<const float *>(rec + 512);
    __syncwarp();
    const signed char *q = s_q[w];
    const float *step = s_step[w];
    float o[8];
    if (lane == 0) {
        level_group(q, step, 3, 0, 0, 0, avg, o);
#pragma unroll
        for (int v = 0; v < 8; ++v) s_l3[w][v] = o[v];
    }
    __syncwarp();
    if (lane < 8) {
        const int i = lane & 1, j = (lane >> 1) & 1, k = lane >> 2;
        level_group(q, step, 2, i, j, k, s_l3[w][i + 2 * j + 4 * k], o);
#pragma unroll
        for (int v = 0; v < 8; ++v) s_l2[w][(2 * i + (v & 1)) + 4 * (2 * j + ((v >> 1) & 1)) + 16 * (2 * k + (v >> 2))] = o[v];
    }
    __syncwarp();
#pragma unroll
    for (int gg = 0; gg < 2; ++gg) {
        const int g = lane + 32 * gg;
        const int i = g & 3, j = (g >> 2) & 3, k = g >> 4;
        level_group(q, step, 1, i, j, k, s_l2[w][i + 4 * j + 16 * k], o);
#pragma unroll
        for (int v = 0; v < 8; ++v) s_v[w][(2 * i + (v & 1)) + 8 * (2 * j + ((v >> 1) & 1)) + 64 * (2 * k + (v >> 2))] = o[v];
    }
    __syncwarp();
    const float *a = s_v[w];
    // elements whose clamped global coordinate lies in this block, per axis [lo, hi)
    int lo[3], hi[3];
    const int org[3] = {ox, oy, oz}, dim[3] = {dx, dy, dz}, n[3] = {nx, ny, nz}, cb[3] = {cbx, cby, cbz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        // clamp(org + e, 0, n - 1) in [8 cb, 8 cb + 8)  <=>  e in [lo, hi)
        const int g0 = 8 * cb[ax], g1 = min(8 * cb[ax] + 8, n[ax]);   // voxels of the block
        int l = g0 - org[ax], h = g1 - org[ax];
        if (g0 == 0) l = 0;                           // elements below the cube map to voxel 0
        if (g1 == n[ax]) h = dim[ax];                 // elements above it map to voxel n - 1
        lo[ax] = max(l, 0);
        hi[ax] = min(h, dim[ax]);
    }
    const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
    if (ex <= 0 || ey <= 0 || ez <= 0) return;
    if (ex == 8 && ey == 8 && ez == 8 && lo[0] == 8 * cbx - ox && lo[1] == 8 * cby - oy && lo[2] == 8 * cbz - oz &&
        8 * cbx + 8 <= nx && 8 * cby + 8 <= ny && 8 * cbz + 8 <= nz) {
        // a block inside the cube whose voxels land once each, unclamped: element lo + v holds
        // voxel v (blocks on an upper face hold padding beyond the cube: generic path)
        float *d0 = dst + ((long long)lo[2] * dy + lo[1]) * dx + lo[0];
#pragma unroll 4
        for (int i = lane; i < 512; i += 32)
            d0[((long long)(i >> 6) * dy + ((i >> 3) & 7)) * dx + (i & 7)] = a[i];
        return;
    }
    const int cnt = ex * ey * ez;
    for (int i = lane; i < cnt; i += 32) {
        const int x = lo[0] + i % ex, y = lo[1] + (i / ex) % ey, z = lo[2] + i / (ex * ey);
        const int gx = clampi(ox + x, 0, nx - 1) - 8 * cbx, gy = clampi(oy + y, 0, ny - 1) - 8 * cby;
        const int gz = clampi(oz + z, 0, nz - 1) - 8 * cbz;
        dst[((long long)z * dy + y) * dx + x] = a[gx + 8 * gy + 64 * gz];
    }
}

}  // namespace

cudaError_t launch_wavelet_encode(const float *cube, int nx, int ny, int nz, unsigned char *store,
                                  cudaStream_t s) {
    const int bnx = (nx + 7) / 8, bny = (ny + 7) / 8, bnz = (nz + 7) / 8;
    const long long nb = (long long)bnx * bny * bnz;
    if (nb <= 0) return cudaSuccess;
    const long long grid = (nb + kWarpsPerCta - 1) / kWarpsPerCta;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_wavelet_encode<<<(unsigned)grid, 32 * kWarpsPerCta, 0, s>>>(cube, nx, ny, nz, bnx, bny, nb, store);
    return cudaGetLastError();
}

cudaError_t launch_wavelet_decode(const unsigned char *store, int nx, int ny, int nz, const int org[3],
                                  const int dim[3], float *dst, cudaStream_t s) {
    const int bnx = (nx + 7) / 8, bny = (ny + 7) / 8;
    int b0[3], nbk[3];
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        const int g0 = std::min(std::max(org[a], 0), n[a] - 1);
        const int g1 = std::min(std::max(org[a] + dim[a] - 1, 0), n[a] - 1);
        b0[a] = g0 / 8;
        nbk[a] = g1 / 8 - b0[a] + 1;
    }
    const long long nbl = (long long)nbk[0] * nbk[1] * nbk[2];
    const long long grid = (nbl + kWarpsPerCta - 1) / kWarpsPerCta;
    if (nbl <= 0) return cudaSuccess;
    k_wavelet_decode<<<(unsigned)grid, 32 * kWarpsPerCta, 0, s>>>(store, nx, ny, nz, bnx, bny, org[0], org[1],
                                                                 org[2], dim[0], dim[1], dim[2], b0[0], b0[1],
                                                                 b0[2], nbk[0], nbk[1], nbl, dst);
    return cudaGetLastError();
}

}  // namespace vr
