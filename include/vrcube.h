/*
 * vrcube.h -- C ABI of libvrcube.so: bricked direct-volume ray casting of a scalar 3D cube on
 * one GB300 GPU (sm_103a), with depth-ordered (sort-last) compositing of the per-brick
 * sub-images into one frame.
 *
 * Method: Hassan, Fluke & Barnes, "Interactive Visualization of the Largest Radioastronomy
 * Cubes" (arXiv:1008.0135).  The calls follow the paper's statement of the rendering problem:
 * Section 2.3 (load a cube or a sub-cube, optional min/max recomputation, colour map sent by the
 * viewer, render requests carrying the transformation and projection matrices), Section 2.4
 * (each part is ray-cast inside its rendering rectangle; ray/box test; early ray termination;
 * MIP output), Section 2.5 (sub-images composited with the associative "over" operator).
 *
 * Conventions shared by every call
 *   - Return value: VR_OK (0) on success, a negative VR_ERR_* status otherwise.  A failed call
 *     leaves the context usable; vr_error_string() names the status.  No C++ exception leaves
 *     the library: a host memory allocation that fails inside any call returns VR_ERR_OOM, any
 *     other host-side exception VR_ERR_STATE (vr_last_error_message() gives its text).
 *   - Ownership: the caller owns every buffer it passes.  The library copies voxels, tables and
 *     camera parameters into its own storage before returning and never keeps caller pointers.
 *   - Geometry: a cube of nx*ny*nz voxels is stored x fastest: index = x + nx*(y + ny*z).
 *     World units are voxels; voxel (x,y,z) sits at (x+0.5, y+0.5, z+0.5), so the volume box is
 *     [0,nx] x [0,ny] x [0,nz].  Sampling between voxel centres is trilinear, clamped to the
 *     edge at the border.
 *   - Images: width W, height H, row 0 at the top, pixel (col i, row j) at flat index j*W + i.
 *     DVR output is premultiplied RGBA float32 (4 floats per pixel) over a transparent black
 *     background; MIP output is one float32 per pixel (the maximum sampled value, vmin where
 *     the ray has no sample).
 *   - Streams: rendering calls are ordered on the CUDA stream passed in (NULL = the legacy
 *     default stream).  Loading and bricking calls are synchronous with respect to the host.
 *   - Threads: one context must not be used by two host threads at once.
 *   - Device: every call makes the context's device current on the calling thread.
 */
#ifndef VRCUBE_H
#define VRCUBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define VR_OK 0
#define VR_ERR_ARG (-1)       /* invalid argument (sizes, ids, null pointers, ranges) */
#define VR_ERR_OOM (-2)       /* device or pinned host allocation failed */
#define VR_ERR_CUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define VR_ERR_TIMEOUT (-4)   /* a bounded wait (brick copy, admission) ran out */
#define VR_ERR_STATE (-5)     /* call out of order (no bricking / table / camera set yet) */
#define VR_ERR_NOT_FOUND (-6) /* unknown cube id */
#define VR_ERR_UNSUPPORTED (-7) /* valid call, combination not offered (e.g. MIP backward) */
#define VR_ERR_IO (-8)          /* a brick source failed (host-side generator or reader) */

/* element / storage types */
#define VR_F32 0
#define VR_F16 1
#define VR_BF16 2
/* buffer locations */
#define VR_HOST 0
#define VR_DEVICE 1
/* projections */
#define VR_ORTHO 0
#define VR_PERSP 1
/* render modes */
#define VR_DVR 0
#define VR_MIP 1
/* early-termination scope (vr_set_termination) */
#define VR_TERM_SEGMENT 0
#define VR_TERM_GLOBAL 1

typedef struct vr_ctx vr_ctx;

/* Cumulative counters since vr_create or the last vr_reset_stats. */
typedef struct {
    int64_t frames;              /* vr_render_frame calls completed */
    int64_t samples;             /* lattice samples evaluated (DVR: composited samples) */
    int64_t fragments;           /* brick x pixel sub-image entries written */
    int64_t bricks_drawn;        /* bricks in the frames' work-lists (not culled) */
    int64_t bricks_sampled;      /* of those, bricks where at least one ray took a sample */
    int64_t brick_bytes_sampled; /* stored bytes (voxels incl. ghost) of the sampled bricks */
    double ms_raycast;           /* device time of the ray-cast kernels (timing enabled) */
    double ms_composite;         /* device time of the compositing kernels (timing enabled) */
    double ms_frame;             /* device time from work-list upload to composite end */
    int64_t timed_frames;        /* frames that carried timing events */
    int64_t bytes_streamed;      /* brick bytes the residency cache received (host copies, or
                                    decoded on the device for compressed cubes) */
    int64_t cache_hits;          /* brick lookups served from the HBM cache */
    int64_t cache_misses;        /* brick lookups that needed a copy or a decode */
    int64_t kernel_errors;       /* bit 0: a staged ray cast gave up waiting for a slab's copies
                                    (its bounded wait ran out; those samples read global memory) */
} vr_stats;

/* Creates a context on CUDA device `device`.  cache_bytes bounds the HBM brick cache used for
 * cubes whose bricks are streamed from host memory (0 = no streaming cache).  *out receives
 * the context; it is released by vr_destroy.  Errors: VR_ERR_ARG (null out, bad device),
 * VR_ERR_CUDA, VR_ERR_OOM. */
int vr_create(vr_ctx **out, int device, size_t cache_bytes);

/* Waits for the context's outstanding work, then frees everything it owns.  NULL is a no-op. */
void vr_destroy(vr_ctx *ctx);

/* Loads a cube (Section 2.3: "the whole cube or a manually specified sub-cube").
 * voxels: nx*ny*nz elements of `dtype` (VR_F32 only) in host (VR_HOST) or device (VR_DEVICE)
 *   memory, x fastest.
 * sub_origin / sub_extent: optional (both NULL or both set) voxel box [origin, origin+extent)
 *   inside the given array; the loaded cube has the extent's dimensions.
 * cube_id: receives the new cube's id.  The voxels are copied; the cube has no bricking yet.
 *   A device source is read after all work already queued on the device (the call
 *   synchronises the device first), so writes still in flight on the caller's streams land.
 * Errors: VR_ERR_ARG (null pointers, non-positive sizes, box outside the array, dtype),
 *   VR_ERR_OOM, VR_ERR_CUDA. */
int vr_load_cube(vr_ctx *ctx, const void *voxels, int dtype, int64_t nx, int64_t ny, int64_t nz,
                 int where, const int64_t *sub_origin, const int64_t *sub_extent, int *cube_id);

/* Creates a streamed cube whose voxels are generated on demand, brick by brick, on host
 * threads: the stand-in for cubes larger than HBM (Section 1.2: HIPASS 12 GB, GASS 25 GB,
 * ASKAP-size cubes of terabytes).  Voxel (x,y,z) = hash noise + Gaussian sources, defined by:
 *   SplitMix64 (state += 0x9E3779B97F4A7C15; two xor-shift-multiply rounds; final xor-shift);
 *   noise: counter c = (z*ny + y)*ceil(nx/2) + floor(x/2), h = SplitMix64 of c ^ (seed *
 *   0xD1B54A32D192ED03), u1 = ((h>>40) + 0.5) 2^-24, u2 = ((h>>16) & 0xFFFFFF) 2^-24,
 *   r = sqrt(-2 ln u1), even x: r cos(2 pi u2), odd x: r sin(2 pi u2) (Box-Muller);
 *   sources: 4 per 256^3 cell q = (qz*ncy + qy)*ncx + qx from the SplitMix64 stream seeded
 *   with seed ^ (q * 0x9E3779B97F4A7C15) ^ 0x632BE59BD9B4E019, six uniforms (top 53 bits)
 *   each: centre (q + u) 256, sigma_xy = 1 + 3u, sigma_z = sigma_xy (2 + 3u), amplitude
 *   exp(ln 3 + (ln 100 - ln 3) u); a source adds amp exp(-r^2/2) inside |dx|,|dy| <= 4 sigma_xy,
 *   |dz| <= 4 sigma_z, d measured from the voxel centre;
 *   voxel = (float)(noise + sources in increasing (cell, k) order), computed in double.
 * The cube must be bricked (vr_set_bricking) before rendering.  Frames stream the bricks they
 * need through the context's HBM brick cache (cache_bytes of vr_create, LRU, pinned staging,
 * copies on a side stream); frames needing more bricks than the cache holds are ray-cast in
 * chunks.  The cache cuts its memory into slots of the largest brick it has seen; a frame
 * whose bricks are larger re-cuts it (dropping its contents) once no serving frame holds a
 * slot, else the frame returns VR_ERR_UNSUPPORTED.  Not offered for streamed cubes: min/max,
 * update, backward, no-allocation frames.
 * Errors: VR_ERR_ARG (null, sizes < 1 or > 2^30). */
int vr_load_cube_procedural(vr_ctx *ctx, uint64_t seed, int64_t nx, int64_t ny, int64_t nz,
                            int *cube_id);

/* Test hook: host-side fault injection into the brick streaming path (nothing is injected on
 * the GPU).  kind 0: off; 1: the brick source throws on the after-th brick it produces
 * (the frame fails with VR_ERR_IO); 2: pinned staging allocation fails (VR_ERR_OOM);
 * 3: waits for staging buffers report expiry (VR_ERR_TIMEOUT).  Errors: VR_ERR_ARG. */
int vr_set_fault_injection(vr_ctx *ctx, int kind, int64_t after);

/* Replaces the voxels of a loaded cube (same dimensions, VR_F32, host or device) and rebuilds
 * its bricks with the current bricking.  For fitting loops that update the voxels.  The copy
 * and the rebuild are ordered on `cuda_stream` and the call returns once they are done.
 * Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND, VR_ERR_CUDA. */
int vr_update_cube(vr_ctx *ctx, int cube_id, const void *voxels, int where, void *cuda_stream);

/* Frees a cube and its bricks.  Errors: VR_ERR_NOT_FOUND. */
int vr_free_cube(vr_ctx *ctx, int cube_id);

/* Exact minimum and maximum of the cube's voxels (Section 2.3: "ask the server to recalculate
 * the cube minimum and maximum").  Synchronous.  Errors: VR_ERR_NOT_FOUND, VR_ERR_CUDA. */
int vr_compute_minmax(vr_ctx *ctx, int cube_id, float *vmin, float *vmax);

/* Splits the cube into a regular grid of bricks of core size bx*by*bz voxels (the last brick
 * along an axis is the remainder) and stores each with `ghost` voxels copied from its
 * neighbours on every side (replicated at the cube border), so the trilinear stencil of every
 * sample a brick owns lies inside that brick (Section 2.2: object-space partitioning; each
 * part is rendered on its own).  storage: VR_F32, VR_F16 or VR_BF16.  16-bit storage keeps,
 * per brick, a power-of-two scale 2^e with e chosen from the brick's stored max |v| (FP16:
 * max|v| 2^-e <= 2^14; BF16: <= 1), the codes being round-to-nearest-even of v 2^-e.
 * Synchronous.  Errors: VR_ERR_ARG (sizes < 1, ghost != 1, storage), VR_ERR_NOT_FOUND,
 * VR_ERR_UNSUPPORTED (slice atlases kept and a brick's atlas beyond the device's 2D-gather
 * size; a compressed cube with a storage other than VR_F32), VR_ERR_OOM, VR_ERR_CUDA. */
int vr_set_bricking(vr_ctx *ctx, int cube_id, int bx, int by, int bz, int ghost, int storage);

/* Lossy wavelet compression of a resident cube (Section 6: wavelet compression of the cube
 * portions kept in GPU memory, with fast decompression and random access, to store and render
 * larger cubes).  The cube's FP32 voxels are encoded into a block store in HBM and then
 * released, with its brick pool and atlases: the cube then renders like a streamed cube, its
 * bricks decoded on demand (on the device) into the brick cache, which must exist (cache_bytes
 * > 0 at vr_create; else frames return VR_ERR_OOM, as for streamed cubes).  Bricking keeps its geometry and becomes
 * VR_F32 (decoded bricks are FP32; other storages return VR_ERR_UNSUPPORTED).
 * Format: the cube is cut into 8x8x8 blocks on a global grid (blocks at the upper faces repeat
 * the edge voxels).  Each block takes three levels of the 3D Haar average/difference transform
 * (s = (a + b)/2, d = (a - b)/2 in binary32, along x then y then z, each level on the previous
 * level's averages); its 511 detail coefficients are rounded (to nearest even) to int8 codes in
 * units of one power-of-two step per subband, the smallest 2^e (-126 <= e <= 120) with
 * max |c| <= 127 2^e over the subband; the block average stays FP32.  One block is a 544-byte
 * record (codes at [0, 512) indexed x + 8 y + 64 z in the pyramid layout, entry 0 unused; the
 * average as FP32 at [512, 516); the 21 steps' exponents as int8 at [516, 537), index
 * 7 (level - 1) + (bx + 2 by + 4 bz) - 1, -128 for an all-zero subband; zeros to 544); records
 * in x-fastest block order: 1.0625 bytes per voxel.  Decoding inverts the transform (a = s + d,
 * b = s - d, along z then y then x, finest level last), so a voxel's error is at most the sum
 * of half a step over the 21 subbands that reach it, plus binary32 rounding.
 * Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND, VR_ERR_UNSUPPORTED (streamed cube), VR_ERR_OOM,
 * VR_ERR_CUDA.  Compressing a compressed cube does nothing. */
int vr_compress_cube(vr_ctx *ctx, int cube_id);

/* The block store of a compressed cube.  dst == NULL: *bytes = its size.  Otherwise copies it
 * into host memory dst of *bytes >= that size (synchronous).  Errors: VR_ERR_ARG,
 * VR_ERR_NOT_FOUND, VR_ERR_STATE (not compressed), VR_ERR_CUDA. */
int vr_wavelet_store(vr_ctx *ctx, int cube_id, void *dst, size_t *bytes);

/* Brick layouts kept for a cube (how the stored bricks of Section 2.2's parts are laid out for
 * the ray caster of Section 2.4).  Bits 0-2 of `mask` keep a copy of every brick whose axis a
 * (0 x, 1 y, 2 z) is the contiguous one in memory; bit 0 is always kept.  Each frame reads the
 * copy whose contiguous axis is most aligned with an image axis and runs its warps along that
 * image axis, so the 32 rays of a warp load neighbouring addresses (each extra layout costs one
 * more copy of the pool in HBM).  Bit 3 also keeps a slice atlas of every brick: a 2D texture
 * array whose tiles are the brick's z-slices, from which a sample's 8 stencil voxels are read
 * by two texture gathers (exact texels; images identical to the linear copies).  When atlases
 * are kept every DVR and MIP frame reads them, and so does the adjoint's replay.  An atlas must
 * fit the device's 2D-gather size (32768 texels a side; 258^3 stored bricks need 8256 x 2322).
 * A bricked cube is rebuilt.  Streamed and compressed cubes (bricks made resident in the brick
 * cache) take mask 1 or 9: with 9, each cache slot holding one of the cube's bricks also holds
 * its slice atlas (a 2D array sized for the cube's largest brick, packed from the slot on the
 * cache's stream when the brick becomes resident).  The arrays of as many slots as the cube
 * has bricks (at most all slots: up to as much device memory again as cache_bytes, outside
 * it) are made by this call (and by vr_set_bricking of such a cube), so that frames only pack; the call
 * then sizes the brick cache (VR_ERR_OOM without one, or when an array cannot be had; a frame
 * that needs another array and cannot have it fails with VR_ERR_OOM too).
 * Bit 4 (resident cubes) keeps, for each kept linear copy, another copy whose rows are padded
 * to 16 bytes; DVR frames of FP32 bricks then stage slabs of each brick in shared memory (bulk
 * copies of those rows) and read the stencils from there (frames identical to the linear
 * copies'; measured slower than the gathers on HIPASS-scale frames, so opt-in),
 * and take precedence over atlases for those frames.
 * Bit 5 (with bit 3; resident cubes of FP16 or BF16 bricks) makes the atlases pair atlases:
 * tile z holds, in 32-bit texels, the codes of slices z and z + 1 side by side, so one gather
 * returns a sample's 8 stencil codes (one texture request per sample instead of two, twice the
 * atlas memory); images are identical to the slice atlases'.  FP32 bricks keep slice atlases.
 * Mask 1..63 with bit 0 set (and bit 3 with bit 5).  Errors: VR_ERR_ARG (mask), VR_ERR_NOT_FOUND, VR_ERR_UNSUPPORTED
 * (streamed or compressed cube with a mask other than 1 or 9; atlas beyond the gather size,
 * raised by the rebuild, or for streamed cubes by the frame), VR_ERR_OOM, VR_ERR_CUDA. */
int vr_set_brick_layouts(vr_ctx *ctx, int cube_id, int mask);

/* Transfer function (Section 2: value -> colour and opacity; Section 2.3: colour map sent by
 * the viewer).  rgba: n x 4 float32 non-premultiplied entries, 2 <= n <= 4096, host memory.
 * A value v maps to u = clamp((v - vmin)/(vmax - vmin), 0, 1), x = u (n-1), and the colour is
 * linear between entries floor(x) and floor(x)+1.  Requires vmax > vmin.  Errors: VR_ERR_ARG. */
int vr_set_transfer_function(vr_ctx *ctx, const float *rgba, int n, float vmin, float vmax);

/* Camera (Section 2.3: "transformation and projection matrices").
 * view: 4x4 row-major world -> eye matrix [R | t] (eye looks down -z, x right, y up).
 * proj: VR_ORTHO (param = image height in world units) or VR_PERSP (param = vertical field of
 * view in radians, 0 < param < pi).  width, height: frame size in pixels (1..16384).
 * The ray of pixel (i, j) goes through the image-plane point of the pixel centre; orthographic
 * rays start on the plane z_eye = 0, perspective rays at the eye.  Only t >= 0 is sampled.
 * Errors: VR_ERR_ARG. */
int vr_set_camera(vr_ctx *ctx, const float view[16], int proj, float param, int width,
                  int height);

/* Render parameters.  mode: VR_DVR or VR_MIP.  step: lattice spacing along the ray in world
 * units (samples at t = k*step, k integer, measured from the ray origin; Section 3 uses a step
 * that samples every voxel a ray crosses at least once).  ert_threshold tau: early ray
 * termination (Section 2.4) stops a brick's segment of a ray once its accumulated opacity
 * reaches tau (test: transmittance <= 1 - tau after compositing a sample); tau >= 1 disables
 * it.  Errors: VR_ERR_ARG (mode, step <= 0, tau <= 0). */
int vr_set_render_params(vr_ctx *ctx, int mode, float step, float ert_threshold);

/* Scope of DVR early ray termination (Section 2.4: a ray stops once its accumulated value
 * reaches its maximum; Section 2.5: the parts' sub-images are composited in depth order).
 * VR_TERM_SEGMENT (default): every brick ray-casts its own segment of a ray from full
 * transmittance and stops it at tau; the bricks' sub-images (fragments) are then composited
 * front to back, so each brick works independently, as on the paper's cluster.
 * VR_TERM_GLOBAL (occlusion skipping): one pass in which every pixel's ray walks the cube's
 * bricks front to back, sampling each brick's segment exactly as the fragment path would (the
 * same samples, owners and arithmetic), carrying one transmittance through them, and stops
 * once the whole ray's opacity reaches tau, so samples behind opaque pixels are skipped.  The
 * image is the unbricked ray's (global termination); it differs from VR_TERM_SEGMENT's by at
 * most 1 - tau per channel.  No fragments are written (stats count none).  Streamed and
 * compressed cubes: the frame's bricks (those the per-segment frame would draw) are made
 * resident in the brick cache together, then walked the same way (VR_ERR_UNSUPPORTED when they
 * do not all fit the cache).  Not available for vr_render_frame_noalloc or vr_render_backward
 * (both VR_ERR_UNSUPPORTED); MIP ignores it.
 * Errors: VR_ERR_ARG. */
int vr_set_termination(vr_ctx *ctx, int mode);

/* Host output mode of vr_render_frame with VR_HOST.  async = 0
 * (the default): the call returns after the frame has been copied into `out`.  async = 1: it
 * returns once the copy into `out` is queued on `cuda_stream`, so that the caller can prepare
 * and queue the next frame while this one renders (an interactive viewer shows frame k - 1
 * while frame k is drawn); the caller synchronises the stream, or an event recorded on it
 * after the call, before it reads `out`, and keeps `out` alive and unchanged until then.  The
 * copy overlaps the host only if `out` is page-locked (e.g. cudaMallocHost); a pageable `out`
 * makes the copy synchronous, as with async = 0.  Frames still run one after another on the
 * stream, and the library's own scratch is reused safely.  Errors: VR_ERR_ARG. */
int vr_set_host_output_async(vr_ctx *ctx, int async);

/* Renders one frame of cube `cube_id` with the current table, camera and parameters.
 * out: W*H*4 floats (DVR) or W*H floats (MIP) in host (VR_HOST) or device (VR_DEVICE) memory.
 * With VR_DEVICE the call returns once the work is queued on `cuda_stream`; with VR_HOST it
 * returns after the frame has been copied into `out` (or once that copy is queued, see
 * vr_set_host_output_async).
 * Steps: per-brick rendering rectangles and culling (host), one ray-cast launch over all
 * (brick, 32x8 or 8x32 pixel tile of its rectangle) work items writing one premultiplied
 * fragment per brick and pixel, one compositing launch blending each pixel's fragments front to
 * back in 16x16 screen tiles (Section 2.5).  With VR_TERM_GLOBAL the two launches are one walk
 * of every pixel's ray through the bricks (see vr_set_termination).
 * Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND, VR_ERR_STATE (no bricking, table or camera),
 * VR_ERR_OOM, VR_ERR_CUDA, VR_ERR_TIMEOUT (streamed bricks did not arrive in time). */
int vr_render_frame(vr_ctx *ctx, int cube_id, float *out, int out_where, void *cuda_stream);

/* Object-space partition (Section 2.2, Fig. 3: each GPU gets a portion of the cube, cut along
 * the current longest axis, and each node cuts its portion again for its GPUs).  After this
 * call frames of the cube draw only the bricks of one part: at level L = 0 .. nlevels-1 the
 * current part's brick grid is cut along its longest axis (in voxels; ties to the lower axis)
 * into counts[L] consecutive slabs of whole brick layers, as even as the layer count allows, and
 * part index[L] is kept (e.g. {3} and {r} for rank r of 3; {2, 2} and {node, gpu} for two
 * nodes of two GPUs).  A part may be empty.  nlevels = 0 restores the whole cube.  The bricking
 * is unchanged (a part's frame samples its bricks exactly as the whole cube's frame does).
 * Global early termination (VR_TERM_GLOBAL) is refused for partitioned cubes: parts terminate
 * per segment, as the paper's nodes do.  Errors: VR_ERR_ARG (nlevels outside 0..8, counts
 * outside 1..65536, index outside 0..counts-1), VR_ERR_NOT_FOUND. */
int vr_set_partition(vr_ctx *ctx, int cube_id, int nlevels, const int *counts, const int *index);

/* How the partition's cuts are placed (Section 3: the slowest GPU sets the frame time, and a
 * part's work depends on the view).  0 (the default): equal layer counts.  1: balanced for the
 * current camera -- each cut falls where the cumulative estimated cost of the part's brick
 * layers crosses k/counts[L] of its total, a brick's cost being the samples a full bundle of
 * the frame's rays takes through it (its window-clipped core volume over a pixel's footprint
 * at its depth times the step; 0 when skipped as empty space or outside the frame; early
 * termination not modelled; computed once per render state and shared by the part's frame and
 * compositing calls).  Balanced parts change with the camera, so every rank needs the
 * whole cube (or the bricks any view can give it); the ranks agree on the cuts because they
 * compute them from the same camera, table and bricking.  The no-allocation renderer refuses
 * balanced partitions (VR_ERR_UNSUPPORTED).  Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND. */
int vr_set_partition_balance(vr_ctx *ctx, int cube_id, int balanced);

/* The brick index range [lo, hi) per axis of the cube's part, and (axes, NULL to skip) the split
 * axis (0 x, 1 y, 2 z) of each partition level.  Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND,
 * VR_ERR_STATE (no bricking). */
int vr_get_partition(vr_ctx *ctx, int cube_id, int lo[3], int hi[3], int *axes);

/* The sub-image of the cube's part (Section 2.5, the frame portion a GPU generates): the frame
 * of vr_render_frame restricted to the part's bricks, with DVR pixels holding premultiplied
 * colour and the TRANSMITTANCE T of the part (not 1 - T: the parts' sub-images compose exactly
 * from (C, T)), and MIP pixels -inf where the part has no sample.  out: W*H*4 (DVR) or W*H
 * (MIP) floats in host or device memory.  DVR needs VR_TERM_SEGMENT.  Errors: as
 * vr_render_frame, VR_ERR_UNSUPPORTED (global termination). */
int vr_render_subimage(vr_ctx *ctx, int cube_id, float *out, int out_where, void *cuda_stream);

/* Second compositing stage (Section 2.5, Fig. 4: the sub-images of sibling parts blended in
 * depth order; the operator is associative, not commutative).  subs: the n = counts[level]
 * sub-images of the sibling parts of `level` (the parts that share every partition index but
 * index[level], in index order), restricted to frame rows [row0, row0 + rows): n * rows * W * 4
 * (DVR, (C, T)) or n * rows * W (MIP) floats, part-major, 16-byte aligned device memory.  Each
 * pixel blends them front to back in the order its ray crosses them: the siblings are
 * consecutive slabs along the level's split axis, crossed in increasing index order when the
 * ray's direction along that axis (the fragment kernel's FP32 ray of the current camera) is
 * positive and in decreasing order when negative.  out: rows * W * 4 (or rows * W) floats,
 * device memory: the parent part's sub-image rows, or, with final != 0, the frame's format
 * (C, 1 - T; MIP -inf becomes vmin).  The camera, mode and table range must be those the
 * sub-images were rendered with.  Ordered on `cuda_stream`.  Errors: VR_ERR_ARG (level outside
 * the partition, n != counts[level], rows outside the frame, misaligned pointers),
 * VR_ERR_NOT_FOUND, VR_ERR_STATE (no bricking or camera), VR_ERR_CUDA. */
int vr_composite_subimages(vr_ctx *ctx, int cube_id, int level, int n, const float *subs, int row0,
                           int rows, int final_, float *out, void *cuda_stream);

/* Renders one frame like vr_render_frame, but allocates no memory at all, for callers that
 * cannot allocate device memory while they render (their GPU memory is owned by another
 * allocator or held to a fixed budget, or their frame loop must not pay the device-wide
 * synchronisation that cudaMalloc/cudaFree can cause).  The paper has no counterpart: this is
 * an operational variant of the Section 2.4/2.5 rendering path.
 * out: device memory, 16-byte aligned, W*H*4 floats (DVR) or W*H floats (MIP); the caller also
 *   supplies the loaded, bricked cube and the current table, camera and parameters.
 * Scratch: the staged work-list and the per-brick fragments live in one static 64 MiB device
 *   array that every GPU loading this library reserves until the process exits.  A frame whose
 *   scratch would exceed 64 MiB is rejected with VR_ERR_ARG (vr_last_error_message() gives the
 *   bytes needed); e.g. 512x512 frames of cubes with a few dozen bricks fit, 1024x1024 frames of
 *   a 12 GB cube do not.  The work-list is built in a static 64 MiB host arena, page-locked in
 *   place (its own pages; nothing is allocated) so that its upload is asynchronous.
 * Set-up: the first call in the process page-locks the host arena; the first call on a device
 *   looks up that array's device address (cudaGetSymbolAddress with the device current), which
 *   may also load the library's GPU code on that device, and creates one event there.  Make
 *   that first call before any stream capture.
 * Sharing: every call, from any context, uses the same array and leaves its contents behind;
 *   calls whose GPU work overlaps (e.g. on two streams without ordering between them) race on
 *   it and corrupt each other's frames.  Calls ordered on one stream are safe.  Host calls are
 *   serialised by a lock.
 * Returns when the work is queued on `cuda_stream`.  The host arena holds one work-list: a call
 * first waits until the previous call's upload has run (that upload waits only for the work
 * queued before it on its stream), at most 60 s (VR_ERR_TIMEOUT).  Errors: VR_ERR_ARG (null or
 * misaligned out, frame too large for the scratch), VR_ERR_NOT_FOUND, VR_ERR_STATE,
 * VR_ERR_UNSUPPORTED (streamed cubes, which need the brick cache; DVR with VR_TERM_GLOBAL),
 * VR_ERR_TIMEOUT, VR_ERR_CUDA. */
int vr_render_frame_noalloc(vr_ctx *ctx, int cube_id, float *out, void *cuda_stream);

/* Gradient of a scalar image loss L with respect to the transfer-function table and the
 * voxels, for the current camera, table and parameters (DVR only, VR_F32 bricks).
 * grad_out: W*H*4 floats dL/d(output RGBA), device memory.
 * grad_lut: n*4 floats, device memory, overwritten with dL/d(table).
 * grad_voxels: nx*ny*nz floats, device memory, dL/d(voxel) ADDED to its contents (NULL: skip).
 * The forward fragments are those of the last vr_render_frame when no call that can change a
 * frame (cube, bricking, table, camera, parameters, termination, mask, window) came between
 * it and this call, else they are recomputed; each ray segment is then replayed front to back
 * from its stored final colour and transmittance (no per-sample state is kept).  The early
 * termination stops of the forward pass are held fixed.  Ordered on `cuda_stream`.
 * Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND, VR_ERR_STATE, VR_ERR_UNSUPPORTED (MIP or 16-bit
 * bricks), VR_ERR_OOM, VR_ERR_CUDA. */
int vr_render_backward(vr_ctx *ctx, int cube_id, const float *grad_out, float *grad_lut,
                       float *grad_voxels, void *cuda_stream);

/* One view of a batch: the row-major world -> eye matrix, projection and its parameter (as in
 * vr_set_camera; every view of a batch has the current camera's width and height). */
typedef struct vr_view {
    float view[16];
    int proj;
    float param;
} vr_view;

/* Gradient of a scalar loss over a batch of views (the fitting loop's render-many-views step)
 * with respect to the table and the voxels, as vr_render_backward for each view in turn, with
 * the table gradients of all views summed in FP64 on the device and rounded to FP32 once.
 * views: n_views cameras; grad_out: n_views * H * W * 4 floats (view-major), device memory,
 * 16-byte aligned; grad_lut: n*4 floats, device memory, overwritten with the batch's dL/d(table);
 * grad_voxels: as for vr_render_backward (ADDED to; NULL: skip).  The views are replayed last to
 * first, so the last view reuses the fragments of the last vr_render_frame when that frame was
 * of the same camera and nothing else changed; the context's camera is the first view's
 * afterwards.  Every view is validated before any work is queued.  Ordered on `cuda_stream`.
 * Errors: as vr_render_backward. */
int vr_render_backward_views(vr_ctx *ctx, int cube_id, int n_views, const vr_view *views,
                             const float *grad_out, float *grad_lut, float *grad_voxels,
                             void *cuda_stream);

/* Spectral channels (Section 2.3: "enabling/disabling spectral channel(s), which are handled in
 * the same manner" as a colour-map change).  mask[z] = 0 switches channel z of the rendered
 * cube off: its voxels take the value vmin of the transfer function (the bottom of the table
 * range) in place of their data, for DVR, MIP and the gradient (which they then do not
 * receive).  n must equal the cube's nz at render time; mask NULL or n = 0 switches every
 * channel on.  The mask is copied.  Errors: VR_ERR_ARG. */
int vr_set_channel_mask(vr_ctx *ctx, const unsigned char *mask, int64_t n);

/* Render window (Section 2.3: the whole cube or a sub-cube): every ray is clipped to the voxel
 * box [lo, hi) (world coordinates, intersected with the cube) with the same slab decisions as
 * the bricks; voxels outside still feed the trilinear stencils at the window's faces.
 * lo = hi = NULL removes the window.  Errors: VR_ERR_ARG (hi <= lo on an axis). */
int vr_set_window(vr_ctx *ctx, const int64_t lo[3], const int64_t hi[3]);

/* Enables (1) or disables (0) device timing of every frame's phases (CUDA events on the frame's
 * stream, read by vr_get_stats).  Errors: VR_ERR_ARG. */
int vr_set_timing(vr_ctx *ctx, int enable);

/* Debug switch: full_rect = 1 launches every brick over the whole frame instead of its
 * rendering rectangle, and keeps bricks that empty-space skipping would drop (a DVR brick whose
 * stored value range maps only to table entries of zero opacity adds exactly nothing).
 * Section 2.4 states such optimisation steps do not change the image; tests use this switch to
 * check it.  Errors: VR_ERR_ARG. */
int vr_set_full_rect(vr_ctx *ctx, int full_rect);

/* Copies the counters (waits for the context's outstanding frames).  Errors: VR_ERR_ARG. */
int vr_get_stats(vr_ctx *ctx, vr_stats *stats);

/* Zeroes the counters.  Errors: VR_ERR_ARG. */
int vr_reset_stats(vr_ctx *ctx);

/* Brick grid of a cube: number of bricks per axis and the storage type.  Errors: VR_ERR_ARG,
 * VR_ERR_NOT_FOUND, VR_ERR_STATE (no bricking). */
int vr_get_brick_grid(vr_ctx *ctx, int cube_id, int64_t nbricks[3], int *storage);

/* Copies brick `brick` (index cx + nbx*(cy + nby*cz)) as stored: its stored dimensions dims[3]
 * (core + 2*ghost per axis), its global voxel origin org[3] (index of stored element (0,0,0),
 * i.e. core origin - ghost), its scale exponent *exp2 (0 for VR_F32), and, when data != NULL,
 * its elements (dims product x 4 bytes for VR_F32, x 2 bytes for 16-bit codes) into host
 * memory.  Errors: VR_ERR_ARG, VR_ERR_NOT_FOUND, VR_ERR_STATE, VR_ERR_CUDA. */
int vr_get_brick(vr_ctx *ctx, int cube_id, int64_t brick, int dims[3], int org[3], int *exp2,
                 void *data);

/* ----------------------------------------------------------------------------------------- */
/* Serving: an interactive request loop with continuous batching                             */
/* ----------------------------------------------------------------------------------------- */
typedef struct {
    int cube_id;
    float view[16];              /* as vr_set_camera */
    int proj;
    float param;
    int width, height;
    int mode;                    /* as vr_set_render_params */
    float step, ert_threshold;
    const float *lut;            /* n x 4 host table, read when the request is admitted */
    int nlut;
    float vmin, vmax;
    double arrival_ms;           /* arrival time, ms after the loop starts (non-decreasing) */
    float *out;                  /* caller's frame buffer (device or pinned host memory) */
    int out_where;               /* VR_DEVICE or VR_HOST */
    int termination;             /* as vr_set_termination: VR_TERM_SEGMENT (0) or VR_TERM_GLOBAL */
} vr_request;

typedef struct {
    int status;                  /* VR_OK or this request's error */
    double admit_ms, done_ms;    /* ms after the loop starts */
    double latency_ms;           /* completion - arrival */
} vr_request_result;

typedef struct {
    int max_inflight;            /* frame slots (streams with their own scratch), 1..64 */
} vr_serve_config;

typedef struct {
    int64_t completed, failed;
    double wall_ms;              /* loop start to last completion */
    double p50_ms, p99_ms, max_ms;  /* latency percentiles of the completed requests */
    double frames_per_s;
    int max_concurrent;          /* most frames in flight at once */
} vr_serve_summary;

/* Serves `n` requests that arrive at their arrival times (the paper's server answering render
 * requests, Section 2.3, with many viewers): requests that have arrived are admitted, in
 * arrival order, as soon as a frame slot is free and -- for streamed cubes -- the brick cache
 * holds enough slots that no frame in flight needs for the bricks the request still lacks (a
 * request needing more than the whole cache runs alone, in chunks).  Admitted frames run
 * concurrently, one CUDA stream per slot; each result equals what vr_render_frame gives for
 * the same request (with its termination scope; a global-termination frame of a streamed cube
 * whose bricks exceed the cache fails alone with VR_ERR_UNSUPPORTED).  Blocks until every request has completed or failed.  res[i] receives
 * request i's status and times; sum (nullable) the latency percentiles and throughput.
 * Host outputs should be pinned (a pageable copy serialises the loop).  Errors: VR_ERR_ARG
 * (null, max_inflight, unordered arrivals, request without table or output),
 * VR_ERR_NOT_FOUND (cube), VR_ERR_STATE (some request failed: see res[i].status). */
int vr_serve(vr_ctx *ctx, const vr_request *reqs, int n, const vr_serve_config *cfg,
             vr_request_result *res, vr_serve_summary *sum);

/* The same loop as an online server a viewer submits to while frames run (the paper's server
 * waiting for render requests, Section 2.3): vr_serve_open starts the loop on a host thread of
 * its own; vr_serve_submit hands it one request, which arrives at that moment (its arrival_ms
 * is ignored); vr_serve_poll returns finished requests; vr_serve_close waits for every submitted
 * request, stops the thread and frees the server.  Admission, concurrency and results are
 * those of vr_serve.  While a server is open its context's cubes must not be loaded, freed,
 * re-bricked or partitioned, and no other call may use the context.  Should the loop stop on a
 * host-side exception (e.g. host memory exhausted), it waits for its frames in flight, every
 * request it holds finishes with VR_ERR_STATE, and later submissions return VR_ERR_STATE. */
typedef struct vr_server vr_server;

/* cfg->max_inflight frame slots (1..64).  *out: the server (owned by the library until
 * vr_serve_close).  Errors: VR_ERR_ARG, VR_ERR_CUDA, VR_ERR_OOM. */
int vr_serve_open(vr_ctx *ctx, const vr_serve_config *cfg, vr_server **out);

/* Submits one request; the table is copied now, `out` must stay valid until the request's
 * ticket is returned by vr_serve_poll (or the server is closed).  *ticket: its number, 0, 1, 2,
 * ... in submission order.  Thread-safe.  Errors: VR_ERR_ARG (null, no table or output),
 * VR_ERR_NOT_FOUND (cube), VR_ERR_STATE (the server is closing). */
int vr_serve_submit(vr_server *srv, const vr_request *req, int64_t *ticket);

/* Up to `cap` finished requests, in completion order: tickets[k] and results[k] (status, times
 * in ms after vr_serve_open, latency from submission to completion); *n how many.  Waits up to
 * wait_ms (0..60000) for the first one when none is ready.  Thread-safe.  Errors: VR_ERR_ARG. */
int vr_serve_poll(vr_server *srv, int64_t *tickets, vr_request_result *results, int cap, int *n,
                  int wait_ms);

/* Waits until every submitted request has finished, stops the loop and frees the server;
 * results not yet polled are dropped.  sum (nullable): percentiles and throughput of all its
 * requests.  Errors: VR_ERR_ARG; VR_ERR_STATE when some request failed. */
int vr_serve_close(vr_server *srv, vr_serve_summary *sum);

/* Name of a status code (static string). */
const char *vr_error_string(int status);

/* Detail of the last failure on the calling thread (which call or CUDA error), "" if none.
 * The string stays valid until the thread's next failing call. */
const char *vr_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* VRCUBE_H */
