// vr_bricks.cu -- cube-level kernels: exact min/max, brick gather with ghost voxels, and the
// 16-bit brick encoding with a per-brick power-of-two scale.
//
// Bricking follows the object-space partition of Section 2.2 (each part rendered on its own);
// the ghost layer makes every trilinear stencil of a sample a brick owns local to that brick.
#include <algorithm>

#include "vr_internal.cuh"

namespace vr {
namespace {

// Monotone map of float bits to unsigned ints (so atomicMin/atomicMax order floats exactly).
__device__ __forceinline__ unsigned int f2ord(float x) {
    unsigned int b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_minmax(const float *__restrict__ v, long long n, unsigned int *enc) {
    unsigned int lo = 0xffffffffu, hi = 0u;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned int e = f2ord(__ldg(v + i));
        lo = min(lo, e);
        hi = max(hi, e);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(enc, lo);
        atomicMax(enc + 1, hi);
    }
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// max |v|, min and max over each brick's stored region (core + ghost, clamped to the cube):
// maxbits[b] (float bits), and range[2b], range[2b+1] (order-preserving encodings).
__global__ void k_brick_maxabs(const float *__restrict__ cube, int nx, int ny, int nz,
                               const DrawBrick *__restrict__ bricks, unsigned int *maxbits,
                               unsigned int *range) {
    const DrawBrick &b = bricks[blockIdx.y];
    int x0 = max(b.org[0], 0), x1 = min(b.org[0] + b.dim[0], nx);
    int y0 = max(b.org[1], 0), y1 = min(b.org[1] + b.dim[1], ny);
    int z0 = max(b.org[2], 0), z1 = min(b.org[2] + b.dim[2], nz);
    int rows = (y1 - y0) * (z1 - z0);
    float m = 0.0f, lo = INFINITY, hi = -INFINITY;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        int y = y0 + r % (y1 - y0), z = z0 + r / (y1 - y0);
        const float *row = cube + ((long long)z * ny + y) * nx;
        for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
            const float v = __ldg(row + x);
            m = fmaxf(m, fabsf(v));
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxbits + blockIdx.y, __float_as_uint(m));
        atomicMin(range + 2 * blockIdx.y, f2ord(lo));
        atomicMax(range + 2 * blockIdx.y + 1, f2ord(hi));
    }
}

// ceil(log2 m) from the exact frexp decomposition; FP16 keeps 14 bits of headroom below 2^15.
__device__ __forceinline__ int scale_exponent(float m, int storage) {
    if (!(m > 0.0f)) return 0;
    int e;
    float f = frexpf(m, &e);
    int cl = (f == 0.5f) ? e - 1 : e;
    return storage == 1 ? cl - 14 : cl;
}

template <int S>
__global__ void k_brick_build(const float *__restrict__ cube, int nx, int ny, int nz,
                              const DrawBrick *__restrict__ bricks,
                              const unsigned int *__restrict__ maxbits, void *pool, int *exps) {
    const DrawBrick &b = bricks[blockIdx.y];
    int e = 0;
    if (S != 0) e = scale_exponent(__uint_as_float(maxbits[blockIdx.y]), S);
    if (S != 0 && blockIdx.x == 0 && threadIdx.x == 0) exps[blockIdx.y] = e;
    int dx = b.dim[0], dy = b.dim[1], dz = b.dim[2];
    int rows = dy * dz;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        int ly = r % dy, lz = r / dy;
        int gy = clampi(b.org[1] + ly, 0, ny - 1), gz = clampi(b.org[2] + lz, 0, nz - 1);
        const float *src = cube + ((long long)gz * ny + gy) * nx;
        // the brick's layout decides the strides (x need not be the contiguous axis)
        const long long dst = b.data_off + (long long)ly * b.str[1] + (long long)lz * b.str[2];
        for (int lx = threadIdx.x; lx < dx; lx += blockDim.x) {
            float v = __ldg(src + clampi(b.org[0] + lx, 0, nx - 1));
            const long long o = dst + (long long)lx * b.str[0];
            if (S == 0) {
                static_cast<float *>(pool)[o] = v;
            } else if (S == 1) {
                static_cast<__half *>(pool)[o] = __float2half_rn(ldexpf(v, -e));
            } else {
                static_cast<__nv_bfloat16 *>(pool)[o] = __float2bfloat16_rn(ldexpf(v, -e));
            }
        }
    }
}

}  // namespace

cudaError_t launch_minmax(const float *v, long long n, unsigned int *enc, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    int grid = (int)(blocks < 152 * 16 ? (blocks > 0 ? blocks : 1) : 152 * 16);
    k_minmax<<<grid, 256, 0, s>>>(v, n, enc);
    return cudaGetLastError();
}

cudaError_t launch_brick_maxabs(const float *cube, int nx, int ny, int nz, const DrawBrick *bricks,
                                int nbricks, unsigned int *maxbits, unsigned int *range,
                                cudaStream_t s) {
    if (nbricks <= 0) return cudaSuccess;
    dim3 grid(64, nbricks);
    k_brick_maxabs<<<grid, 256, 0, s>>>(cube, nx, ny, nz, bricks, maxbits, range);
    return cudaGetLastError();
}

// Slice atlas: element (x, y, z) of the x-contiguous brick goes to atlas column
// (z & (2^alog - 1)) dx + x, row (z >> alog) dy + y.  Raw bits are moved (codes stay codes).
template <typename T>
__global__ void k_atlas_pack(const T *__restrict__ src, int dx, int dy, int dz, int alog, char *atlas,
                             size_t pitch) {
    const long long n = (long long)dx * dy * dz;
    const int cm = (1 << alog) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % dx);
        const long long r = i / dx;
        const int y = (int)(r % dy), z = (int)(r / dy);
        const size_t row = (size_t)(z >> alog) * dy + y, col = (size_t)(z & cm) * dx + x;
        reinterpret_cast<T *>(atlas + row * pitch)[col] = src[i];
    }
}

// The same placement written straight into the atlas array through a surface (no staging, no
// array copy).  Coordinates are in range by construction; the zero boundary mode makes any
// write outside the array a no-op rather than a fault.
template <typename T>
__global__ void k_atlas_pack_surf(const T *__restrict__ src, int dx, int dy, int dz, int alog,
                                  cudaSurfaceObject_t surf) {
    const long long n = (long long)dx * dy * dz;
    const int cm = (1 << alog) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % dx);
        const long long r = i / dx;
        const int y = (int)(r % dy), z = (int)(r / dy);
        const int row = (z >> alog) * dy + y, col = (z & cm) * dx + x;
        surf2Dwrite<T>(src[i], surf, col * (int)sizeof(T), row, cudaBoundaryModeZero);
    }
}

cudaError_t launch_atlas_pack_surf(const void *brick, int esz, int dx, int dy, int dz, int alog,
                                   unsigned long long surf, cudaStream_t s) {
    const long long n = (long long)dx * dy * dz;
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    if (esz == 4)
        k_atlas_pack_surf<unsigned int><<<grid, 256, 0, s>>>(static_cast<const unsigned int *>(brick), dx, dy, dz,
                                                             alog, (cudaSurfaceObject_t)surf);
    else
        k_atlas_pack_surf<unsigned short><<<grid, 256, 0, s>>>(static_cast<const unsigned short *>(brick), dx, dy,
                                                               dz, alog, (cudaSurfaceObject_t)surf);
    return cudaGetLastError();
}

cudaError_t launch_atlas_pack(const void *brick, int esz, int dx, int dy, int dz, int alog, void *atlas,
                              size_t pitch, cudaStream_t s) {
    const long long n = (long long)dx * dy * dz;
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    if (esz == 4)
        k_atlas_pack<unsigned int><<<grid, 256, 0, s>>>(static_cast<const unsigned int *>(brick), dx, dy, dz,
                                                        alog, static_cast<char *>(atlas), pitch);
    else
        k_atlas_pack<unsigned short><<<grid, 256, 0, s>>>(static_cast<const unsigned short *>(brick), dx, dy,
                                                          dz, alog, static_cast<char *>(atlas), pitch);
    return cudaGetLastError();
}

// Pair atlas of a 16-bit brick: texel (x, y) of tile z (z < dz - 1), placed at column
// (z & (2^alog - 1)) dx + x, row (z >> alog) dy + y, holds the code of element (x, y, z) in its
// low half and that of (x, y, z + 1) in its high half.
__device__ __forceinline__ void pair_texel(const unsigned short *src, int dx, int dy, int dz, int alog, long long i,
                                           unsigned int &val, int &col, int &row) {
    const int x = (int)(i % dx);
    const long long r = i / dx;
    const int y = (int)(r % dy), z = (int)(r / dy);
    const size_t e = ((size_t)z * dy + y) * dx + x;
    val = (unsigned int)src[e] | ((unsigned int)src[e + (size_t)dx * dy] << 16);
    col = (z & ((1 << alog) - 1)) * dx + x;
    row = (z >> alog) * dy + y;
}

__global__ void k_pair_pack(const unsigned short *__restrict__ src, int dx, int dy, int dz, int alog, char *atlas,
                            size_t pitch) {
    const long long n = (long long)dx * dy * (dz - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned int v;
        int col, row;
        pair_texel(src, dx, dy, dz, alog, i, v, col, row);
        reinterpret_cast<unsigned int *>(atlas + (size_t)row * pitch)[col] = v;
    }
}

// The same through a surface (zero boundary mode: a write outside the array is a no-op).
__global__ void k_pair_pack_surf(const unsigned short *__restrict__ src, int dx, int dy, int dz, int alog,
                                 cudaSurfaceObject_t surf) {
    const long long n = (long long)dx * dy * (dz - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned int v;
        int col, row;
        pair_texel(src, dx, dy, dz, alog, i, v, col, row);
        surf2Dwrite<unsigned int>(v, surf, col * (int)sizeof(unsigned int), row, cudaBoundaryModeZero);
    }
}

cudaError_t launch_pair_pack(const void *brick, int dx, int dy, int dz, int alog, void *atlas, size_t pitch,
                             unsigned long long surf, cudaStream_t s) {
    const long long n = (long long)dx * dy * (dz - 1);
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    if (surf)
        k_pair_pack_surf<<<grid, 256, 0, s>>>(static_cast<const unsigned short *>(brick), dx, dy, dz, alog,
                                              (cudaSurfaceObject_t)surf);
    else
        k_pair_pack<<<grid, 256, 0, s>>>(static_cast<const unsigned short *>(brick), dx, dy, dz, alog,
                                         static_cast<char *>(atlas), pitch);
    return cudaGetLastError();
}

cudaError_t launch_brick_build(const float *cube, int nx, int ny, int nz, const DrawBrick *bricks,
                               int nbricks, const unsigned int *maxbits, int storage, void *pool,
                               int *exps, cudaStream_t s) {
    if (nbricks <= 0) return cudaSuccess;
    dim3 grid(64, nbricks);
    if (storage == 0)
        k_brick_build<0><<<grid, 256, 0, s>>>(cube, nx, ny, nz, bricks, maxbits, pool, exps);
    else if (storage == 1)
        k_brick_build<1><<<grid, 256, 0, s>>>(cube, nx, ny, nz, bricks, maxbits, pool, exps);
    else
        k_brick_build<2><<<grid, 256, 0, s>>>(cube, nx, ny, nz, bricks, maxbits, pool, exps);
    return cudaGetLastError();
}

}  // namespace vr
