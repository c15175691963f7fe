// vr_host.h -- host-side state of libvrcube.so shared by its translation units (context, cubes,
// per-frame work-lists, error reporting).  Not part of the public ABI (include/vrcube.h is).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <new>
#include <stdexcept>
#include <vector>

#include "vr_internal.cuh"
#include "../../include/vrcube.h"

namespace vrh {

using namespace vr;

// Detail of the last failure on this thread (vr_last_error_message).
inline thread_local std::string g_last_error;

inline int cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
}
inline int arg_fail(const char *what) {
    g_last_error = what;
    return VR_ERR_ARG;
}
inline int fail(int status, const std::string &what) {
    g_last_error = what;
    return status;
}

// No C++ exception crosses the C ABI: every entry point runs its body through abi_guard, which
// turns a host allocation failure into VR_ERR_OOM and any other host-side exception into
// VR_ERR_STATE (vr_last_error_message gives its text).
inline int abi_fail(int status, const char *what) noexcept {
    try {
        g_last_error = what;
    } catch (...) {
    }
    return status;
}
template <class F>
inline int abi_guard(F &&body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return abi_fail(VR_ERR_OOM, "host memory allocation failed");
    } catch (const std::length_error &) {
        return abi_fail(VR_ERR_OOM, "host allocation size out of range");
    } catch (const std::exception &e) {
        return abi_fail(VR_ERR_STATE, e.what());
    } catch (...) {
        return abi_fail(VR_ERR_STATE, "unexpected host-side exception");
    }
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return vrh::cuda_fail(e_, #call); \
    } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct BrickCache;   // HBM brick cache of streamed cubes (vr_residency.cu)

struct Cube {
    int64_t n[3] = {0, 0, 0};
    float *d_src = nullptr;           // FP32 source voxels, x fastest (resident cubes)
    bool bricked = false;
    int B[3] = {0, 0, 0};
    int ghost = 1;
    int storage = VR_F32;
    int64_t nb[3] = {0, 0, 0};
    std::vector<DrawBrick> tmpl;      // one record per brick (geometry, pool offsets, exponent)
    DrawBrick *d_tmpl = nullptr;      // device copy used by the build kernels
    void *d_pool = nullptr;
    size_t pool_bytes = 0;
    unsigned int *d_bs = nullptr;     // per brick: max |v| bits, exponent, min, max (4 words)
    std::vector<float> vlo, vhi;      // per-brick value range of the stored region
    // brick layouts kept in the pool: bit a = a copy whose axis a is contiguous (x always kept);
    // bit 3 = a slice-atlas texture of every brick besides the pool
    int layouts = 1;
    std::vector<long long> loff;      // element offset of brick b in layout a: loff[3 b + a]
    // layout bit 4: each kept linear copy again with its rows padded to 16 bytes (staged frames
    // copy rows of it into shared memory): offset of brick b's padded copy along a
    std::vector<long long> loff_pad;
    std::vector<cudaArray_t> atlas_arr;          // per brick (layout bit 3)
    std::vector<unsigned long long> atlas_tex;   // texture objects over them
    size_t atlas_bytes = 0;
    bool atlas_pair = false;           // the atlases are pair atlases (layout bit 5, 16-bit bricks)
    // streamed cubes: bricks are produced on the host and cached in HBM on demand
    bool streamed = false;
    // compressed cubes (also `streamed`): 8x8x8 wavelet blocks in HBM, bricks decoded on demand
    bool wavelet = false;
    unsigned char *d_wstore = nullptr;
    size_t wstore_bytes = 0;
    uint64_t proc_seed = 0;           // procedural cube: generator seed
    int id = 0;
    // object-space partition (Section 2.2): frames draw only the bricks of one part of a
    // recursive longest-axis split; part_nlev = 0 draws the whole cube
    static constexpr int kMaxPartLevels = 8;
    int part_nlev = 0;
    int part_counts[kMaxPartLevels] = {0};
    int part_index[kMaxPartLevels] = {0};
    int part_balance = 0;             // 1: cuts balanced by the current camera's estimated cost
    // balanced cuts: every brick's estimated cost for the render state it was computed in
    // (cost_key = the context's state_gen - part_gen then; partition calls change neither)
    mutable std::vector<double> cost_cache;
    mutable uint64_t cost_key = ~0ull;
};

// The part of a cube's brick grid that its partition selects: brick index ranges [lo, hi) per
// axis and the split axis of every level (the longest axis, in voxels, of the parent part).
struct PartBox {
    int lo[3], hi[3];
    int axis[Cube::kMaxPartLevels];
};
PartBox partition_box(const vr_ctx *c, const Cube *cb);
bool in_part(const PartBox &p, const Cube *cb, int64_t brick);

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;                   // elements
};

struct WorkList {
    std::vector<DrawBrick> db;
    std::vector<TileItem> items;
    std::vector<int> tile_start, tile_list;
    long long frag_px = 0;
    // offsets inside the staged upload
    size_t off_lut = 0, off_db = 0, off_items = 0, off_ts = 0, off_tl = 0, off_mask = 0, bytes = 0;
};

}  // namespace vrh

struct vr_ctx {
    int device = 0;
    cudaStream_t load_stream = nullptr;
    std::map<int, vrh::Cube *> cubes;
    int next_id = 1;
    // transfer function (copied into every frame's upload)
    std::vector<float4> lut;
    float vmin = 0.0f, vmax = 1.0f;
    bool tf_set = false;
    // camera
    vr::Cam cam{};
    bool cam_set = false;
    // render parameters
    int mode = VR_DVR;
    float step = 0.5f;
    float tau = 0.99f;
    int term = VR_TERM_SEGMENT;       // early termination per brick segment or global (waves)
    bool full_rect = false;
    bool subimage = false;            // the frame being rendered is a part's sub-image (C, T)
    bool timing = false;
    // Section 2.3 viewer controls: spectral channels switched off, sub-cube window
    std::vector<unsigned char> chmask;   // per cube z; empty = every channel on
    bool has_window = false;
    int64_t win_lo[3] = {0, 0, 0}, win_hi[3] = {0, 0, 0};
    // frame scratch (reused; guarded by events)
    char *h_stage = nullptr;
    size_t h_cap = 0;
    vrh::DevBuf<char> d_stage;
    vrh::DevBuf<char> d_frags;        // bytes
    vrh::DevBuf<float4> d_gfrag;
    vrh::DevBuf<float> d_gpart;
    vrh::DevBuf<double> d_gacc;         // FP64 table-gradient sum over the views of a batch
    vrh::DevBuf<double> d_gchunk;       // FP64 chunk sums of a view's table-gradient partials
    vrh::DevBuf<float> d_out;
    cudaEvent_t upload_done = nullptr, frame_done = nullptr;
    bool frame_pending = false;
    vr::Counters *d_ctr = nullptr;
    unsigned int *d_mm = nullptr;     // min/max scratch (2 ordered-bit words)
    // statistics
    int64_t frames = 0, fragments = 0, bricks_drawn = 0, timed_frames = 0;
    double ms_raycast = 0, ms_composite = 0, ms_frame = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::vector<cudaEvent_t>> ev_pending;
    // streamed cubes
    size_t cache_bytes = 0;
    vrh::BrickCache *cache = nullptr;
    bool async_host_out = false;      // serving slots: no host sync after a VR_HOST copy
    int fault_kind = 0;               // host-side fault injection (tests)
    int64_t fault_after = -1;
    // d_frags holds the DVR fragments of cube frag_cube for render state state_gen: every call
    // that can change a frame bumps state_gen; every other write of d_frags clears frag_valid.
    // vr_render_backward reuses them instead of ray-casting the frame again.
    uint64_t state_gen = 0, frag_gen = 0;
    uint64_t part_gen = 0;            // the state_gen bumps made by partition calls
    int frag_cube = -1;
    bool frag_valid = false;
};

namespace vrh {

// Per-frame choice of brick layout and warp orientation.  Linear copies: the one whose
// contiguous world axis is most aligned with an image axis, and warps running along that image
// axis, so the 32 rays of a warp load neighbouring addresses.  Slice atlases (when kept, always
// preferred): warps along the image axis closer to the z-slices' plane, so a warp's gathers
// stay within few slices; the linear copy for kernels that read linear bricks follows the
// same image axis.
struct FrameLayout {
    int layout;                       // contiguous world axis of the linear copy (0 x, 1 y, 2 z)
    int lanes_y;                      // warps along image y (1) or image x (0)
    int tw, th;                       // ray-cast tile size in pixels
    float align;                      // |cos| between that image axis and the contiguous axis
    int atlas;                        // 1: the ray caster gathers from the slice atlases
};
FrameLayout frame_layout(const vr_ctx *c, const Cube *cb);
// Strides of the copy of a dim[0] x dim[1] x dim[2] brick whose axis a is contiguous, its rows
// padded to a multiple of 16 bytes (esz-byte elements); returns the copy's elements.
long long layout_strides_padded(const int dim[3], int a, int esz, int str[3]);
// Empty-space skipping: prefix counts of table entries with non-zero opacity, and whether a
// brick's value range reaches only zero-opacity entries (its fragment would be a no-op).
void alpha_prefix(const vr_ctx *c, std::vector<int> &pre);
bool skip_brick(const vr_ctx *c, const Cube *cb, size_t b, const int *pre);
void layout_strides(const int dim[3], int layout, int str[3]);
// The brick grid a global-termination frame walks (the render window clips the rays).
MarchGrid march_grid(const vr_ctx *c, const Cube *cb);

int set_dev(vr_ctx *c);
Cube *find_cube(vr_ctx *c, int id);
int ensure_host(vr_ctx *c, size_t bytes);
void eye_f32(const Cam &c, float o[3]);
void build_worklist(vr_ctx *c, Cube *cb, WorkList &wl);
FrameConsts make_consts(vr_ctx *c, Cube *cb);
int timing_events(vr_ctx *c, cudaEvent_t ev[4]);

// The timing events of one frame (vr_set_timing): taken from the context's pool, handed to
// the pending list once the frame is queued, and put back in the pool by the destructor when
// the frame fails before that.
struct FrameTiming {
    vr_ctx *c;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool queued = false;
    explicit FrameTiming(vr_ctx *ctx) : c(ctx) {}
    FrameTiming(const FrameTiming &) = delete;
    FrameTiming &operator=(const FrameTiming &) = delete;
    ~FrameTiming() {
        if (!queued)        // a failed timing_events may have taken only some of the four
            for (auto e : ev)
                if (e) c->ev_pool.push_back(e);
    }
    void queue() {
        if (ev[0]) c->ev_pending.push_back({ev[0], ev[1], ev[2], ev[3]});
        queued = true;
    }
};
int collect_timing(vr_ctx *c);
int stage_frame(vr_ctx *c, Cube *cb, WorkList &wl, cudaStream_t s, cudaEvent_t ev0);
int check_ready(vr_ctx *c, Cube *cb);
// Core box of brick b clipped to the render window; false when nothing of it is left.
bool window_clip(const vr_ctx *c, const Cube *cb, const DrawBrick &b, float lo[3], float hi[3]);
int build_bricks(vr_ctx *c, Cube *cb, cudaStream_t s);
int render_frame_impl(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s);
void free_cube(Cube *cb);

template <typename T>
int ensure(DevBuf<T> &b, size_t n, vr_ctx *c) {
    if (b.cap >= n && b.p) return VR_OK;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    size_t want = n > b.cap * 3 / 2 ? n : b.cap * 3 / 2;
    if (b.p) CK(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
    CK(cudaMalloc(&b.p, (want > 0 ? want : 1) * sizeof(T)));
    b.cap = want;
    return VR_OK;
}

// residency (vr_residency.cu)
int cache_create(vr_ctx *c);
void cache_destroy(vr_ctx *c);
int render_streamed(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s);
int render_streamed_global(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s);
void cache_stats(vr_ctx *c, vr_stats *st);
void cache_reset_stats(vr_ctx *c);
void cache_forget_cube(vr_ctx *c, int cube_id);
int streamed_brick(Cube *cb, int64_t brick, void *data, int *exp2);
size_t cache_slot_bytes(vr_ctx *c);   // 0 until the cache has been sized
int cache_prepare_atlases(vr_ctx *c, Cube *cb);   // slot atlases for a cube with layout bit 3
// admission accounting of the serving loop: bricks of a work-list not yet resident and the
// cache slots no in-flight frame holds (VR_ERR_TIMEOUT while another frame is making bricks
// resident), and holding / releasing a frame's bricks (false if busy and !wait)
int cache_missing(vr_ctx *c, Cube *cb, const WorkList &wl, int64_t *missing, int64_t *free_slots);
bool cache_hold(vr_ctx *c, Cube *cb, const std::vector<int64_t> &bricks, int delta, bool wait);
int streamed_exp(Cube *cb, int64_t brick, int *exp2);

}  // namespace vrh
