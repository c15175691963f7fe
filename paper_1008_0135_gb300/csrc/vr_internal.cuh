// vr_internal.cuh -- types and launchers shared by the translation units of libvrcube.so.
// Nothing here is part of the public ABI (include/vrcube.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace vr {

constexpr int kTile = 16;          // compositing: 16x16 screen tiles
constexpr int kRcLong = 32;        // ray-cast work item: 32x8 (or 8x32) pixels of a rectangle,
constexpr int kRcShort = 8;        // one warp per 32-pixel row (or column)
constexpr int kMaxLut = 4096;      // transfer-function entries (float4 each) held in shared memory

// Camera constants in the FP32 decision arithmetic (computed once per frame on the host).
struct Cam {
    float R[9];                    // rows of the view rotation (world -> eye)
    float t[3];                    // view translation
    float half_w, half_h;          // orthographic half extents of the image plane
    float th_w, th;                // perspective: tan(fov/2) * aspect, tan(fov/2)
    int proj, W, H;
};

struct FrameConsts {
    Cam cam;
    float step;                    // lattice spacing along the ray
    float thr;                     // early-termination transmittance threshold 1 - tau (>= 0)
    float vmin, inv_range;         // table mapping u = (v - vmin) * inv_range
    float lutmax;                  // n - 1
    int nlut;
    int mode;                      // 0 DVR, 1 MIP
    int storage;                   // 0 f32, 1 f16, 2 bf16
    int nx, ny, nz;                // cube size
    int lanes_y;                   // 0: a warp's 32 lanes run along image x (tiles 32x8);
                                   // 1: along image y (tiles 8x32)
    int fetch;                     // how a sample's 8 stencil corners are read: 0 = 8 loads from
                                   // the linear brick, 1 = the same with the stencil cache (rays
                                   // keep shared corners; poorly aligned layout), 2 = 2 gathers
                                   // from the brick's slice-atlas texture, 4 = slabs of the
                                   // brick staged in shared memory by bulk copies from the copy
                                   // with 16-byte rows (DVR, FP32 bricks), 5 = 1 gather from
                                   // the brick's pair atlas (16-bit bricks)
    const unsigned char *chmask;   // per spectral channel (cube z): 0 = disabled; null = none
    int sub;                       // 1: a part's sub-image -- DVR pixels keep the transmittance T
                                   // (not 1 - T), MIP pixels without samples stay -inf
    int stage_m, stage_dir;        // fetch 4: the march axis the slabs are staged along (the
                                   // view's dominant axis other than the contiguous one) and the
                                   // direction the rays cross it (+1 / -1)
};

// One brick of the current frame's work-list (front-to-back order).
struct DrawBrick {
    float lo[3], hi[3];            // core box [lo, hi) in world units
    float org_c[3];                // stored origin + 0.5: local stored coordinate = p - org_c
    int org[3];                    // global voxel index of stored element (0,0,0)
    int dim[3];                    // stored dimensions (core + 2 ghost)
    int str[3];                    // element strides of x, y, z in the stored array (layout)
    int exp2;                      // power-of-two scale exponent (0 for f32)
    int rect[4];                   // x0, y0, w, h of the rendering rectangle (pixels)
    int brick;                     // brick index in the cube's grid
    int sampled;                   // set by the ray-cast kernel when a ray sampled this brick
    long long data_off;            // element offset of the stored brick in the pool
    long long frag_off;            // fragment offset (pixels) of the brick's sub-image
    long long bytes;               // stored bytes of the brick
    unsigned long long atlas;      // texture object over the brick's slice atlas (0: none): a 2D
                                   // array whose tile (z & (2^alog - 1), z >> alog) of dim[0] x
                                   // dim[1] texels holds stored slice z (FP32 values or 16-bit codes)
    int alog;
    int skip;                      // global termination: every sample of this brick adds nothing
                                   // (its values map only to zero opacity), walk through it
    long long pad_off;             // staged frames (fetch 4): element offset of the brick's copy
    int pad_str[3];                // with 16-byte rows (the frame layout's contiguous axis) and
                                   // its strides; -1 when the cube keeps no such copy
};

// The brick grid a global-termination frame walks: nb bricks per axis of core size B over a
// cube of size n (voxels; the last brick along an axis holds the remainder), rays clipped to
// [clo, chi) (the cube, or the render window inside it).
struct MarchGrid {
    int nb[3];
    float B[3], n[3];
    float invB[3];                 // 1 / B (rounded): a first guess of a cell, settled exactly
    float clo[3], chi[3];
};

struct TileItem {                  // one ray-cast work item
    int db;                        // DrawBrick index
    int tx, ty;                    // 16x16 tile inside the brick's rectangle
};

struct Counters {                  // device-side cumulative counters
    unsigned long long samples;
    unsigned long long brick_bytes_sampled;
    unsigned long long bricks_sampled;
    unsigned long long pad;
};

// ---------------------------------------------------------------------------------------------
// launchers (return cudaError_t of the launch)
// ---------------------------------------------------------------------------------------------
cudaError_t launch_minmax(const float *v, long long n, unsigned int *enc_minmax,
                          cudaStream_t s);
cudaError_t launch_brick_maxabs(const float *cube, int nx, int ny, int nz, const DrawBrick *bricks,
                                int nbricks, unsigned int *maxbits, unsigned int *range,
                                cudaStream_t s);
// Packs one x-contiguous stored brick (dx*dy*dz elements of esz = 4 or 2 bytes) into a
// pitch-linear slice atlas of (2^alog dx) x (ceil(dz / 2^alog) dy) elements, row pitch `pitch` bytes.
cudaError_t launch_atlas_pack(const void *brick, int esz, int dx, int dy, int dz, int alog, void *atlas,
                              size_t pitch, cudaStream_t s);
cudaError_t launch_atlas_pack_surf(const void *brick, int esz, int dx, int dy, int dz, int alog,
                                   unsigned long long surf, cudaStream_t s);
// Packs one x-contiguous 16-bit brick into its pair atlas (dz - 1 tiles of dx x dy 32-bit
// texels, placed like the slice atlas's tiles): through surface `surf` when non-zero, else into
// the pitch-linear `atlas` of row pitch `pitch` bytes.
cudaError_t launch_pair_pack(const void *brick, int dx, int dy, int dz, int alog, void *atlas, size_t pitch,
                             unsigned long long surf, cudaStream_t s);
cudaError_t launch_brick_build(const float *cube, int nx, int ny, int nz, const DrawBrick *bricks,
                               int nbricks, const unsigned int *maxbits, int storage, void *pool,
                               int *exps, cudaStream_t s);
cudaError_t launch_raycast(const FrameConsts &fc, const float4 *lut, const DrawBrick *db,
                           const TileItem *items, int nitems, const void *pool, void *frags,
                           Counters *ctr, cudaStream_t s);
// Wavelet block store: one record of kWaveletRecordBytes per 8x8x8 block of the cube, blocks
// in x-fastest order over a ceil(n/8) grid (format in vr_wavelet.cu).
constexpr int kWaveletRecordBytes = 544;
cudaError_t launch_wavelet_encode(const float *cube, int nx, int ny, int nz, unsigned char *store,
                                  cudaStream_t s);
// Decodes the stored region of one brick (global voxels clamp(org + [0, dim)), x-contiguous
// FP32) from the block store.
cudaError_t launch_wavelet_decode(const unsigned char *store, int nx, int ny, int nz, const int org[3],
                                  const int dim[3], float *dst, cudaStream_t s);
// Global early termination: every pixel's ray walks the brick grid front to back in one
// launch; premultiplied RGBA into out (W*H float4).  bricks: every brick of the cube in grid
// order (x fastest), with the frame's layout offsets, atlases and skip flags.
cudaError_t launch_raymarch(const FrameConsts &fc, const float4 *lut, DrawBrick *bricks, const MarchGrid &g,
                            const void *pool, float4 *out, Counters *ctr, cudaStream_t s);
cudaError_t launch_composite(const FrameConsts &fc, const DrawBrick *db, const int *tile_start,
                             const int *tile_list, const void *frags, float *out, cudaStream_t s);
// Second-stage compositing of n sibling parts' sub-images (Section 2.5): rows [row0, row0 + rows)
// of the frame, subs = n sub-images of those rows (part-major; DVR (C, T) float4, MIP float),
// blended per pixel in the order its ray crosses the parts along `axis` (parts are consecutive
// slabs along it).  final: write the frame's format ((C, 1 - T); MIP -inf -> vmin).
cudaError_t launch_composite_parts(const FrameConsts &fc, int axis, int n, const float *subs, int row0, int rows,
                                   int final_, float *out, cudaStream_t s);
cudaError_t launch_composite_backward(const FrameConsts &fc, const DrawBrick *db,
                                      const int *tile_start, const int *tile_list,
                                      const float4 *frags, const float4 *gout, float4 *gfrag,
                                      cudaStream_t s);
cudaError_t launch_adjoint(const FrameConsts &fc, const float4 *lut, const DrawBrick *db,
                           const TileItem *items, int nitems, const float *pool,
                           const float4 *frags, const float4 *gfrag, float *glut_partial,
                           float *gvox, cudaStream_t s);
// The table gradient from the adjoint's per-CTA partials (nparts x 4 nlut floats), summed in
// FP64 through `chunks` (kLutGradChunks x 4 nlut doubles of scratch): glut = the sum; with
// several views, acc (4 nlut doubles) = (first ? 0 : acc) + the view's sum, and
// glut = (float)acc after the last view.
constexpr int kLutGradChunks = 64;
cudaError_t launch_lut_grad_reduce(const float *partial, int nparts, int nlut, double *chunks, float *glut,
                                   cudaStream_t s);
cudaError_t launch_lut_grad_accumulate(const float *partial, int nparts, int nlut, double *chunks, double *acc,
                                       bool first, cudaStream_t s);
cudaError_t launch_lut_grad_store(const double *acc, int nlut, float *glut, cudaStream_t s);

}  // namespace vr
