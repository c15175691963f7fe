// vr_residency.cu -- bricks of cubes larger than HBM: produced on host threads (here by the
// procedural cube generator), staged in pinned host buffers, copied to HBM on a side stream,
// and kept in an LRU cache of fixed-size brick slots.
//
// The paper's answer to larger-than-memory cubes (Section 1.2) is to spread the parts over many
// GPUs; on one GPU the same object-space parts become bricks that stream through HBM.  A frame
// whose bricks do not all fit in the cache is ray-cast in chunks: each chunk's bricks are made
// resident, its (brick, tile) items are ray-cast into the frame's fragment buffer, and the
// compositing pass runs once over all fragments (sort-last compositing does not care in which
// order the fragments were produced).
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <atomic>
#include <cstring>
#include <deque>
#include <functional>
#include <future>
#include <mutex>
#include <memory>
#include <stdexcept>
#include <thread>
#include <unordered_map>

#include "vr_host.h"

namespace vrh {

// ---------------------------------------------------------------------------------------------
// procedural cube: hash noise + Gaussian sources (the same definition as the test oracle's
// generator; both follow the published SplitMix64 and Box-Muller definitions)
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kCell = 256;          // source cell size
constexpr int kSrcPerCell = 4;

inline uint64_t sm64_next(uint64_t &st) {
    uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct PSrc {
    double cx, cy, cz, sxy, sz, amp;
};

void cell_sources(uint64_t seed, int64_t qx, int64_t qy, int64_t qz, int64_t ncx, int64_t ncy,
                  PSrc *out) {
    const uint64_t q = (uint64_t)((qz * ncy + qy) * ncx + qx);
    uint64_t st = seed ^ (q * 0x9E3779B97F4A7C15ULL) ^ 0x632BE59BD9B4E019ULL;
    for (int k = 0; k < kSrcPerCell; ++k) {
        double u[6];
        for (int i = 0; i < 6; ++i) u[i] = (double)(sm64_next(st) >> 11) * 0x1.0p-53;
        out[k].cx = ((double)qx + u[0]) * kCell;
        out[k].cy = ((double)qy + u[1]) * kCell;
        out[k].cz = ((double)qz + u[2]) * kCell;
        out[k].sxy = 1.0 + 3.0 * u[3];
        out[k].sz = out[k].sxy * (2.0 + 3.0 * u[4]);
        out[k].amp = std::exp(std::log(3.0) + (std::log(100.0) - std::log(3.0)) * u[5]);
    }
}

// Box-Muller pair of the hashed counter of voxel pair (x >> 1) in row (y, z).
inline void noise_pair(uint64_t seed, int64_t nx, int64_t ny, int64_t xp, int64_t y, int64_t z,
                       double &n_even, double &n_odd) {
    uint64_t st = (uint64_t)((z * ny + y) * ((nx + 1) / 2) + xp) ^ (seed * 0xD1B54A32D192ED03ULL);
    const uint64_t h = sm64_next(st);
    const double u1 = ((double)(h >> 40) + 0.5) * 0x1.0p-24;
    const double u2 = (double)((h >> 16) & 0xFFFFFFULL) * 0x1.0p-24;
    const double r = std::sqrt(-2.0 * std::log(u1));
    const double th = 6.283185307179586 * u2;
    n_even = r * std::cos(th);
    n_odd = r * std::sin(th);
}

// Contribution of a source to voxel (x, y, z); false when outside its +-4 sigma box.
inline bool source_term(const PSrc &s, int64_t x, int64_t y, int64_t z, double &t) {
    const double dx = ((double)x + 0.5) - s.cx, dy = ((double)y + 0.5) - s.cy, dz = ((double)z + 0.5) - s.cz;
    if (!(std::fabs(dx) <= 4.0 * s.sxy && std::fabs(dy) <= 4.0 * s.sxy && std::fabs(dz) <= 4.0 * s.sz)) return false;
    t = s.amp * std::exp(-0.5 * (dx * dx / (s.sxy * s.sxy) + dy * dy / (s.sxy * s.sxy) + dz * dz / (s.sz * s.sz)));
    return true;
}

// FP32 voxels of the box [org, org + dim) with coordinates clamped to the cube, x fastest.
void gen_region(uint64_t seed, const int64_t n[3], const int org[3], const int dim[3], float *out) {
    const int64_t nc[3] = {(n[0] + kCell - 1) / kCell, (n[1] + kCell - 1) / kCell, (n[2] + kCell - 1) / kCell};
    int64_t lo[3], hi[3], qlo[3], qhi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = std::max<int64_t>(org[a], 0);
        hi[a] = std::min<int64_t>((int64_t)org[a] + dim[a] - 1, n[a] - 1);
        // sources reach at most 4 sigma_z <= 80 voxels from their centre, inside their cell
        qlo[a] = std::max<int64_t>(0, (lo[a] - 82) / kCell);
        qhi[a] = std::min<int64_t>(nc[a] - 1, (hi[a] + 82) / kCell);
    }
    std::vector<PSrc> src;
    for (int64_t qz = qlo[2]; qz <= qhi[2]; ++qz)          // increasing cell index q
        for (int64_t qy = qlo[1]; qy <= qhi[1]; ++qy)
            for (int64_t qx = qlo[0]; qx <= qhi[0]; ++qx) {
                PSrc s[kSrcPerCell];
                cell_sources(seed, qx, qy, qz, nc[0], nc[1], s);
                src.insert(src.end(), s, s + kSrcPerCell);
            }
    const int64_t w = hi[0] - lo[0] + 1;
    std::vector<double> row((size_t)w);
    for (int lz = 0; lz < dim[2]; ++lz) {
        const int64_t z = std::min<int64_t>(std::max<int64_t>((int64_t)org[2] + lz, 0), n[2] - 1);
        for (int ly = 0; ly < dim[1]; ++ly) {
            const int64_t y = std::min<int64_t>(std::max<int64_t>((int64_t)org[1] + ly, 0), n[1] - 1);
            for (int64_t x = lo[0]; x <= hi[0];) {
                double ne, no;
                noise_pair(seed, n[0], n[1], x >> 1, y, z, ne, no);
                if ((x & 1) == 0) {
                    row[x - lo[0]] = ne;
                    if (x + 1 <= hi[0]) row[x + 1 - lo[0]] = no;
                    x += 2;
                } else {
                    row[x - lo[0]] = no;
                    x += 1;
                }
            }
            for (const PSrc &s : src) {               // in increasing (cell, k) order
                if (!(std::fabs(((double)y + 0.5) - s.cy) <= 4.0 * s.sxy &&
                      std::fabs(((double)z + 0.5) - s.cz) <= 4.0 * s.sz))
                    continue;
                const int64_t x0 = std::max<int64_t>(lo[0], (int64_t)std::floor(s.cx - 4.0 * s.sxy) - 1);
                const int64_t x1 = std::min<int64_t>(hi[0], (int64_t)std::ceil(s.cx + 4.0 * s.sxy) + 1);
                for (int64_t x = x0; x <= x1; ++x) {
                    double t;
                    if (source_term(s, x, y, z, t)) row[x - lo[0]] += t;
                }
            }
            float *o = out + ((size_t)lz * dim[1] + ly) * dim[0];
            for (int lx = 0; lx < dim[0]; ++lx) {
                const int64_t x = std::min<int64_t>(std::max<int64_t>((int64_t)org[0] + lx, 0), n[0] - 1);
                o[lx] = (float)row[x - lo[0]];
            }
        }
    }
}

// The scale exponent of a 16-bit region whose max |v| is m (FP16 keeps max|v| 2^-e <= 2^14,
// BF16 <= 1).
int region_exponent(float m, int storage) {
    if (!(m > 0.0f)) return 0;
    int ex;
    const float f = std::frexp(m, &ex);
    const int cl = (f == 0.5f) ? ex - 1 : ex;
    return storage == VR_F16 ? cl - 14 : cl;
}

float max_abs(const float *v, size_t count) {
    float m = 0.0f;
    for (size_t i = 0; i < count; ++i) m = std::max(m, std::fabs(v[i]));
    return m;
}

// Round-to-nearest-even 16-bit codes of v 2^-e.
void encode_codes(const float *v, size_t count, int storage, int e, void *codes) {
    if (storage == VR_F16) {
        __half *h = static_cast<__half *>(codes);
        for (size_t i = 0; i < count; ++i) h[i] = __float2half_rn(std::ldexp(v[i], -e));
    } else {
        __nv_bfloat16 *h = static_cast<__nv_bfloat16 *>(codes);
        for (size_t i = 0; i < count; ++i) h[i] = __float2bfloat16_rn(std::ldexp(v[i], -e));
    }
}

// 16-bit codes of a generated FP32 region: the scale exponent from the region's max |v|, then
// the codes.
int encode_region(const float *v, size_t count, int storage, void *codes) {
    const int e = region_exponent(max_abs(v, count), storage);
    encode_codes(v, count, storage, e, codes);
    return e;
}

// ---------------------------------------------------------------------------------------------
// a small pool of host worker threads
// ---------------------------------------------------------------------------------------------
class Workers {
  public:
    explicit Workers(int n) {
        for (int i = 0; i < n; ++i) th_.emplace_back([this] { run(); });
    }
    ~Workers() {
        {
            std::lock_guard<std::mutex> l(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    std::future<void> submit(std::function<void()> f) {
        auto task = std::make_shared<std::packaged_task<void()>>(std::move(f));
        std::future<void> fut = task->get_future();
        {
            std::lock_guard<std::mutex> l(mu_);
            q_.push_back([task] { (*task)(); });
        }
        cv_.notify_one();
        return fut;
    }
    int size() const { return (int)th_.size(); }

  private:
    void run() {
        for (;;) {
            std::function<void()> f;
            {
                std::unique_lock<std::mutex> l(mu_);
                cv_.wait(l, [this] { return stop_ || !q_.empty(); });
                if (stop_ && q_.empty()) return;
                f = std::move(q_.front());
                q_.pop_front();
            }
            f();
        }
    }
    std::vector<std::thread> th_;
    std::deque<std::function<void()>> q_;
    std::mutex mu_;
    std::condition_variable cv_;
    bool stop_ = false;
};

constexpr double kWaitSeconds = 60.0;   // bound of every host wait on the copy engine

// Polls an event until it completes or the bound expires (VR_ERR_TIMEOUT).
int wait_event(cudaEvent_t e, double seconds) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t r = cudaEventQuery(e);
        if (r == cudaSuccess) return VR_OK;
        if (r != cudaErrorNotReady) return cuda_fail(r, "cudaEventQuery");
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > seconds)
            return fail(VR_ERR_TIMEOUT, "a brick copy did not complete within its time bound");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// the cache
// ---------------------------------------------------------------------------------------------
struct Slot {
    int cube = -1;
    int64_t brick = -1;
    uint64_t lru = 0;
    int exp2 = 0;
    int64_t chunk = -1;               // last chunk (global counter) that uses this slot
    cudaEvent_t last_use = nullptr;   // completes after every ray-cast that read the slot so far
    bool used = false;
    int held = 0;                     // in-flight serving frames that need this brick
    // slice atlas of the slot (cubes whose layout mask asks for atlases): a 2D array sized for
    // the largest brick of its storage kind, created on first use
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    cudaSurfaceObject_t surf = 0;     // packs write the array through it (0: staging + copy)
    int arr_storage = -1, arr_w = 0, arr_h = 0, alog = 0;
    bool atlas_ok = false;            // the atlas holds this slot's brick
};

struct Staging {
    void *host = nullptr;             // pinned
    cudaEvent_t done = nullptr;       // its copy finished
    bool pending = false;
};

struct BrickCache {
    char *d_base = nullptr;
    size_t slot_bytes = 0;            // bytes per slot
    int nslots = 0;
    std::vector<Slot> slots;
    std::unordered_map<uint64_t, int> where;   // (cube, brick) -> slot
    uint64_t tick = 0;
    int64_t chunk_counter = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t copies_done = nullptr;
    std::vector<Staging> stage;
    size_t stage_next = 0;
    Workers *workers = nullptr;
    void *pack_tmp = nullptr;         // pitched staging of atlas packs (on the copy stream)
    size_t pack_bytes = 0;
    int64_t hits = 0, misses = 0, bytes = 0, generated = 0;
    std::recursive_mutex mu;          // frames of the serving loop make bricks resident from
                                      // their own host threads
};

static uint64_t key_of(int cube, int64_t brick) { return ((uint64_t)(uint32_t)cube << 40) | (uint64_t)brick; }

int cache_create(vr_ctx *c) {
    if (c->cache) return VR_OK;
    BrickCache *k = new (std::nothrow) BrickCache();
    if (!k) return VR_ERR_OOM;
    c->cache = k;
    CK(cudaStreamCreateWithFlags(&k->copy, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&k->copies_done, cudaEventDisableTiming));
    const unsigned hw = std::thread::hardware_concurrency();
    k->workers = new Workers((int)std::max(2u, std::min(hw ? hw : 4u, 64u)));
    return VR_OK;
}

void cache_destroy(vr_ctx *c) {
    BrickCache *k = c->cache;
    if (!k) return;
    if (k->copy) cudaStreamSynchronize(k->copy);
    delete k->workers;
    for (auto &s : k->slots) {
        if (s.last_use) cudaEventDestroy(s.last_use);
        if (s.tex) cudaDestroyTextureObject(s.tex);
        if (s.surf) cudaDestroySurfaceObject(s.surf);
        if (s.arr) cudaFreeArray(s.arr);
    }
    for (auto &s : k->stage) {
        if (s.host) cudaFreeHost(s.host);
        if (s.done) cudaEventDestroy(s.done);
    }
    if (k->pack_tmp) cudaFree(k->pack_tmp);
    if (k->d_base) cudaFree(k->d_base);
    if (k->copies_done) cudaEventDestroy(k->copies_done);
    if (k->copy) cudaStreamDestroy(k->copy);
    delete k;
    c->cache = nullptr;
}

size_t cache_slot_bytes(vr_ctx *c) {
    if (!c->cache) return 0;
    std::lock_guard<std::recursive_mutex> l(c->cache->mu);
    return c->cache->slot_bytes;
}

static int cache_size(vr_ctx *c, size_t slot_bytes);

int cache_missing(vr_ctx *c, Cube *cb, const WorkList &wl, int64_t *missing, int64_t *free_slots) {
    int rc = cache_create(c);
    if (rc) return rc;
    BrickCache *k = c->cache;
    std::unique_lock<std::recursive_mutex> l(k->mu, std::try_to_lock);
    if (!l.owns_lock()) return VR_ERR_TIMEOUT;     // a frame is making its bricks resident
    size_t max_bytes = 0;
    for (auto &b : cb->tmpl) max_bytes = std::max(max_bytes, (size_t)b.bytes);
    if ((rc = cache_size(c, max_bytes)) != VR_OK) return rc;
    int64_t miss = 0, fr = 0;
    for (auto &d : wl.db)
        if (k->where.find(key_of(cb->id, d.brick)) == k->where.end()) ++miss;
    for (auto &sl : k->slots)
        if (sl.held == 0) ++fr;
    *missing = miss;
    *free_slots = fr;
    return VR_OK;
}

bool cache_hold(vr_ctx *c, Cube *cb, const std::vector<int64_t> &bricks, int delta, bool wait) {
    BrickCache *k = c->cache;
    if (!k) return true;
    std::unique_lock<std::recursive_mutex> l(k->mu, std::defer_lock);
    if (wait) l.lock();
    else if (!l.try_lock()) return false;
    for (int64_t b : bricks) {
        auto it = k->where.find(key_of(cb->id, b));
        if (it != k->where.end()) k->slots[it->second].held = std::max(0, k->slots[it->second].held + delta);
    }
    return true;
}

void cache_stats(vr_ctx *c, vr_stats *st) {
    if (!c->cache) return;
    std::lock_guard<std::recursive_mutex> l(c->cache->mu);
    st->bytes_streamed = c->cache->bytes;
    st->cache_hits = c->cache->hits;
    st->cache_misses = c->cache->misses;
}

void cache_reset_stats(vr_ctx *c) {
    if (!c->cache) return;
    std::lock_guard<std::recursive_mutex> l(c->cache->mu);
    c->cache->hits = c->cache->misses = c->cache->bytes = 0;
}

void cache_forget_cube(vr_ctx *c, int cube_id) {
    BrickCache *k = c->cache;
    if (!k) return;
    std::lock_guard<std::recursive_mutex> l(k->mu);
    for (int i = 0; i < k->nslots; ++i)
        if (k->slots[i].cube == cube_id) {
            k->where.erase(key_of(cube_id, k->slots[i].brick));
            k->slots[i].cube = -1;
            k->slots[i].brick = -1;
        }
}

// Slots and staging sized for `slot_bytes` bricks (first streamed frame).  A cache whose slots
// are too small for a cube's bricks is re-cut, dropping its contents, once nothing holds a
// slot: its copies and every frame that read a slot are waited for first.  All or nothing: on
// failure everything this call allocated is released and the cache stays unsized.
static int cache_size(vr_ctx *c, size_t slot_bytes) {
    BrickCache *k = c->cache;
    if (k->d_base && k->slot_bytes >= slot_bytes) return VR_OK;
    if (k->d_base) {
        for (auto &s : k->slots)
            if (s.held > 0) return fail(VR_ERR_UNSUPPORTED, "larger bricks than the cache's slots while frames hold bricks");
        CK(cudaStreamSynchronize(k->copy));
        for (auto &s : k->slots) {
            if (s.used) CK(cudaEventSynchronize(s.last_use));
            cudaEventDestroy(s.last_use);
            if (s.tex) cudaDestroyTextureObject(s.tex);
            if (s.surf) cudaDestroySurfaceObject(s.surf);
            if (s.arr) cudaFreeArray(s.arr);
        }
        for (auto &s : k->stage) {
            if (s.pending) CK(cudaEventSynchronize(s.done));
            cudaFreeHost(s.host);
            cudaEventDestroy(s.done);
        }
        cudaFree(k->d_base);
        k->d_base = nullptr;
        k->slot_bytes = 0;
        k->nslots = 0;
        k->slots.clear();
        k->stage.clear();
        k->stage_next = 0;
        k->where.clear();
    }
    if (c->cache_bytes < slot_bytes)
        return fail(VR_ERR_OOM, "cache_bytes of vr_create is smaller than one brick");
    const size_t sb = align_up(slot_bytes, 256);
    const int nslots = (int)(c->cache_bytes / sb);
    std::vector<Staging> stage(std::max(4, 2 * k->workers->size()));
    std::vector<Slot> slots(nslots);
    char *base = nullptr;
    auto undo = [&](int status, const std::string &what) {
        for (auto &s : stage) {
            if (s.host) cudaFreeHost(s.host);
            if (s.done) cudaEventDestroy(s.done);
        }
        for (auto &s : slots)
            if (s.last_use) cudaEventDestroy(s.last_use);
        if (base) cudaFree(base);
        return fail(status, what);
    };
    for (auto &s : stage) {
        if (c->fault_kind == 2) return undo(VR_ERR_OOM, "pinned staging allocation failed (injected)");
        if (cudaMallocHost(&s.host, sb) != cudaSuccess) return undo(VR_ERR_OOM, "pinned staging allocation failed");
        if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) return undo(VR_ERR_CUDA, "event");
    }
    for (auto &s : slots)
        if (cudaEventCreateWithFlags(&s.last_use, cudaEventDisableTiming) != cudaSuccess) return undo(VR_ERR_CUDA, "event");
    if (cudaMalloc(&base, (size_t)nslots * sb) != cudaSuccess) return undo(VR_ERR_OOM, "brick cache allocation failed");
    k->d_base = base;
    k->slot_bytes = sb;
    k->nslots = nslots;
    k->slots = std::move(slots);
    k->stage = std::move(stage);
    return VR_OK;
}

// One brick of a streamed cube produced into pinned memory (FP32 values, or 16-bit codes with
// the brick's exponent in *exp2) by the whole worker pool: its box is cut into z-slabs generated
// in parallel -- a voxel depends only on its coordinates, and a slab's source list keeps the
// cells' order, so the values are those of one pass over the box -- and a 16-bit brick is then
// encoded slab by slab with the exponent of its max |v| over all slabs.  `done` is set once
// every slab has finished (or the first error is recorded in err).
struct BrickJob {
    Cube *cb = nullptr;
    DrawBrick b{};
    void *dst = nullptr;
    int exp2 = 0;                      // the brick's scale exponent (16-bit storage)
    std::string err;                   // the first error of a slab ("" if none)
    Workers *pool = nullptr;
    int nslab = 1;
    std::vector<float> tmp;            // FP32 values of a 16-bit brick
    std::vector<float> slab_max;
    std::atomic<int> left{0};
    std::mutex mu;                     // guards err
    std::promise<void> done;
    std::future<void> finished = done.get_future();

    size_t plane() const { return (size_t)b.dim[0] * b.dim[1]; }
    int z0(int i) const { return (int)((int64_t)b.dim[2] * i / nslab); }
    void fail_with(const char *what) {
        std::lock_guard<std::mutex> l(mu);
        if (err.empty()) err = what;
    }
};

static void job_encode(const std::shared_ptr<BrickJob> &j, int i);

static void job_generate(const std::shared_ptr<BrickJob> &j, int i) {
    try {
        const int z0 = j->z0(i), z1 = j->z0(i + 1);
        int org[3] = {j->b.org[0], j->b.org[1], j->b.org[2] + z0};
        int dim[3] = {j->b.dim[0], j->b.dim[1], z1 - z0};
        float *out = j->cb->storage == VR_F32 ? static_cast<float *>(j->dst) + (size_t)z0 * j->plane()
                                              : j->tmp.data() + (size_t)z0 * j->plane();
        if (dim[2] > 0) gen_region(j->cb->proc_seed, j->cb->n, org, dim, out);
        if (j->cb->storage != VR_F32) j->slab_max[i] = max_abs(out, (size_t)dim[2] * j->plane());
    } catch (const std::exception &e) {
        j->fail_with(e.what());
    }
    if (j->left.fetch_sub(1) != 1) return;
    // the last slab: FP32 bricks (or a failed one) are done; 16-bit bricks are encoded next
    bool failed;
    {
        std::lock_guard<std::mutex> l(j->mu);
        failed = !j->err.empty();
    }
    if (j->cb->storage == VR_F32 || failed) {
        j->exp2 = 0;
        j->done.set_value();
        return;
    }
    float m = 0.0f;
    for (float v : j->slab_max) m = std::max(m, v);
    j->exp2 = region_exponent(m, j->cb->storage);
    j->left.store(j->nslab);
    int k = 1;
    try {
        for (; k < j->nslab; ++k) j->pool->submit([j, k] { job_encode(j, k); });
    } catch (...) {                    // no room to queue a task: encode the rest here
        for (; k < j->nslab; ++k) job_encode(j, k);
    }
    job_encode(j, 0);
}

static void job_encode(const std::shared_ptr<BrickJob> &j, int i) {
    try {
        const int z0 = j->z0(i), z1 = j->z0(i + 1);
        const size_t off = (size_t)z0 * j->plane();
        encode_codes(j->tmp.data() + off, (size_t)(z1 - z0) * j->plane(), j->cb->storage, j->exp2,
                     static_cast<char *>(j->dst) + off * 2);
    } catch (const std::exception &e) {
        j->fail_with(e.what());
    }
    if (j->left.fetch_sub(1) == 1) j->done.set_value();
}

// Starts the production of brick `b` on the pool.  The job (shared with the pool's tasks, so a
// caller that stops waiting leaves nothing they write behind) holds the outcome: `finished`
// completes once every slab is done, then `exp2` and `err` are final.
static std::shared_ptr<BrickJob> produce_brick(Workers *pool, Cube *cb, const DrawBrick &b, void *dst,
                                               bool inject) {
    auto j = std::make_shared<BrickJob>();
    j->cb = cb;
    j->b = b;
    j->dst = dst;
    j->pool = pool;
    if (inject) {                      // a failing brick source (host-side fault injection)
        j->err = "brick source failed (injected)";
        j->done.set_value();
        return j;
    }
    j->nslab = std::max(1, std::min(pool->size(), b.dim[2]));
    if (cb->storage != VR_F32) {
        j->tmp.resize(j->plane() * (size_t)b.dim[2]);
        j->slab_max.assign(j->nslab, 0.0f);
    }
    j->left.store(j->nslab);
    int i = 0;
    try {
        for (; i < j->nslab; ++i) pool->submit([j, i] { job_generate(j, i); });
    } catch (...) {                    // no room to queue a task: generate the rest here
        for (; i < j->nslab; ++i) job_generate(j, i);
    }
    return j;
}

// Slice atlases of cache slots (streamed and compressed cubes whose layout mask has bit 3):
// every brick of a cube uses the tile layout of the cube's largest stored brick (2^alog
// z-slices per atlas row), so any of its bricks fits a slot's array.
struct SlotAtlasGeom {
    int w = 0, h = 0, alog = 0;
};

static int slot_atlas_geom(vr_ctx *c, Cube *cb, SlotAtlasGeom &g) {
    int mx[3] = {0, 0, 0};
    for (auto &b : cb->tmpl)
        for (int a = 0; a < 3; ++a) mx[a] = std::max(mx[a], b.dim[a]);
    int l = 0;
    while ((1ll << (2 * l)) < mx[2]) ++l;
    const long long w = (long long)mx[0] << l, h = (long long)((mx[2] + (1 << l) - 1) >> l) * mx[1];
    int gw = 0, gh = 0;
    CK(cudaDeviceGetAttribute(&gw, cudaDevAttrMaxTexture2DGatherWidth, c->device));
    CK(cudaDeviceGetAttribute(&gh, cudaDevAttrMaxTexture2DGatherHeight, c->device));
    if (w > gw || h > gh) return fail(VR_ERR_UNSUPPORTED, "bricks too large for a slice atlas (2D gather limit)");
    g.w = (int)w;
    g.h = (int)h;
    g.alog = l;
    return VR_OK;
}

// Gives slot `si` an atlas array for cube `cb`'s bricks, creating or replacing it when it has
// another texel type or is too small (after every reader and pending copy of the old one).
static int slot_atlas_alloc(vr_ctx *c, Cube *cb, int si, const SlotAtlasGeom &g) {
    BrickCache *k = c->cache;
    Slot &s = k->slots[si];
    const size_t esz = cb->storage == VR_F32 ? 4 : 2;
    if (!s.arr || s.arr_storage != cb->storage || s.arr_w < g.w || s.arr_h < g.h) {
        if (s.arr) {
            if (s.used) CK(cudaEventSynchronize(s.last_use));
            CK(cudaStreamSynchronize(k->copy));
            cudaDestroyTextureObject(s.tex);
            if (s.surf) cudaDestroySurfaceObject(s.surf);
            cudaFreeArray(s.arr);
            s.tex = 0;
            s.surf = 0;
            s.arr = nullptr;
        }
        const cudaChannelFormatDesc cd =
            esz == 4 ? cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat)
            : cb->storage == VR_F16 ? cudaCreateChannelDescHalf()
                                    : cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned);
        // writable through a surface when the device allows it with gathers, else filled by copies
        bool surf_ok = cudaMallocArray(&s.arr, &cd, (size_t)g.w, (size_t)g.h,
                                       cudaArrayTextureGather | cudaArraySurfaceLoadStore) == cudaSuccess;
        if (!surf_ok) {
            s.arr = nullptr;
            cudaGetLastError();
            if (cudaMallocArray(&s.arr, &cd, (size_t)g.w, (size_t)g.h, cudaArrayTextureGather) != cudaSuccess) {
                s.arr = nullptr;
                cudaGetLastError();
                return fail(VR_ERR_OOM, "slice atlas of a cache slot: cudaMallocArray failed");
            }
        }
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = s.arr;
        cudaTextureDesc td{};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        CK(cudaCreateTextureObject(&s.tex, &rd, &td, nullptr));
        if (surf_ok) CK(cudaCreateSurfaceObject(&s.surf, &rd));
        s.arr_storage = cb->storage;
        s.arr_w = g.w;
        s.arr_h = g.h;
        s.atlas_ok = false;
    }
    return VR_OK;
}

// Packs slot `si`'s brick `b` (already queued into the slot on the copy stream) into the slot's
// atlas on the copy stream.
static int slot_atlas_pack(vr_ctx *c, Cube *cb, int si, const DrawBrick &b, const SlotAtlasGeom &g) {
    BrickCache *k = c->cache;
    Slot &s = k->slots[si];
    const size_t esz = cb->storage == VR_F32 ? 4 : 2;
    int rc = slot_atlas_alloc(c, cb, si, g);
    if (rc != VR_OK) return rc;
    if (s.surf) {
        CK(launch_atlas_pack_surf(k->d_base + (size_t)si * k->slot_bytes, (int)esz, b.dim[0], b.dim[1], b.dim[2],
                                  g.alog, (unsigned long long)s.surf, k->copy));
        s.alog = g.alog;
        s.atlas_ok = true;
        return VR_OK;
    }
    const size_t need = (size_t)g.w * g.h * esz;
    if (k->pack_bytes < need) {
        CK(cudaStreamSynchronize(k->copy));
        if (k->pack_tmp) cudaFree(k->pack_tmp);
        k->pack_tmp = nullptr;
        k->pack_bytes = 0;
        CK(cudaMalloc(&k->pack_tmp, need));
        k->pack_bytes = need;
    }
    const size_t w = (size_t)b.dim[0] << g.alog, h = (size_t)((b.dim[2] + (1 << g.alog) - 1) >> g.alog) * b.dim[1];
    CK(launch_atlas_pack(k->d_base + (size_t)si * k->slot_bytes, (int)esz, b.dim[0], b.dim[1], b.dim[2], g.alog,
                         k->pack_tmp, w * esz, k->copy));
    CK(cudaMemcpy2DToArrayAsync(s.arr, 0, 0, k->pack_tmp, w * esz, w * esz, h, cudaMemcpyDeviceToDevice, k->copy));
    s.alog = g.alog;
    s.atlas_ok = true;
    return VR_OK;
}

// Makes the bricks of wl.db[d0, d1) resident: hits keep their slot, misses get the least
// recently used slot not needed by this chunk, are produced on the workers and copied on the
// cache's stream after the slot's previous reader finished.  Fills data_off / exp2.
static int make_resident(vr_ctx *c, Cube *cb, std::vector<DrawBrick> &db, size_t d0, size_t d1,
                         int64_t chunk) {
    BrickCache *k = c->cache;
    const size_t esz = cb->storage == VR_F32 ? 4 : 2;
    const bool atlas = (cb->layouts & 8) != 0;
    SlotAtlasGeom g;
    int rc = VR_OK;
    if (atlas && (rc = slot_atlas_geom(c, cb, g)) != VR_OK) return rc;
    std::vector<std::pair<size_t, int>> misses;   // (db index, slot)
    for (size_t i = d0; i < d1; ++i) {
        auto it = k->where.find(key_of(cb->id, db[i].brick));
        if (it != k->where.end()) {
            Slot &s = k->slots[it->second];
            s.lru = ++k->tick;
            s.chunk = chunk;
            db[i].data_off = (long long)((size_t)it->second * k->slot_bytes / esz);
            db[i].exp2 = s.exp2;
            db[i].atlas = 0ull;
            if (atlas) {
                if (!s.atlas_ok && (rc = slot_atlas_pack(c, cb, it->second, db[i], g)) != VR_OK) return rc;
                db[i].atlas = s.tex;
                db[i].alog = s.alog;
            }
            k->hits++;
        } else {
            misses.push_back({i, -1});
        }
    }
    if (misses.empty()) return VR_OK;
    // victims: free slots first, then least recently used, never one this chunk uses
    std::vector<int> order;
    order.reserve(k->nslots);
    for (int i = 0; i < k->nslots; ++i)
        if (k->slots[i].chunk != chunk) order.push_back(i);
    std::sort(order.begin(), order.end(), [k](int a, int b) {
        const Slot &sa = k->slots[a], &sb = k->slots[b];
        if ((sa.cube < 0) != (sb.cube < 0)) return sa.cube < 0;
        if ((sa.held > 0) != (sb.held > 0)) return sb.held > 0;
        return sa.lru < sb.lru;
    });
    if (order.size() < misses.size()) return fail(VR_ERR_STATE, "brick cache chunking error");
    for (size_t m = 0; m < misses.size(); ++m) {
        const int si = order[m];
        Slot &s = k->slots[si];
        if (s.cube >= 0) k->where.erase(key_of(s.cube, s.brick));
        s.cube = -1;                  // not valid until its copy is issued
        s.atlas_ok = false;
        s.brick = db[misses[m].first].brick;
        s.chunk = chunk;
        s.lru = ++k->tick;
        misses[m].second = si;
    }
    if (cb->wavelet) {
        // compressed cube: each missing brick is decoded from the HBM block store straight into
        // its slot on the cache's stream, after the slot's previous reader
        for (auto &mi : misses) {
            Slot &s = k->slots[mi.second];
            const DrawBrick &b = db[mi.first];
            if (s.used) CK(cudaStreamWaitEvent(k->copy, s.last_use, 0));
            CK(launch_wavelet_decode(cb->d_wstore, (int)cb->n[0], (int)cb->n[1], (int)cb->n[2], b.org, b.dim,
                                     reinterpret_cast<float *>(k->d_base + (size_t)mi.second * k->slot_bytes),
                                     k->copy));
            s.cube = cb->id;
            s.exp2 = 0;
            k->where[key_of(cb->id, s.brick)] = mi.second;
            db[mi.first].data_off = (long long)((size_t)mi.second * k->slot_bytes / esz);
            db[mi.first].exp2 = 0;
            db[mi.first].atlas = 0ull;
            k->misses++;
            k->bytes += b.bytes;
            if (atlas) {
                if ((rc = slot_atlas_pack(c, cb, mi.second, b, g)) != VR_OK) {
                    k->where.erase(key_of(cb->id, s.brick));
                    s.cube = -1;
                    s.brick = -1;
                    s.chunk = -1;
                    return rc;
                }
                db[mi.first].atlas = s.tex;
                db[mi.first].alog = s.alog;
            }
        }
        return VR_OK;
    }
    // produce in parallel, at most one staging buffer per brick in flight
    const size_t nstage = k->stage.size();
    std::vector<std::shared_ptr<BrickJob>> jobs(misses.size());
    std::vector<size_t> st_of(misses.size());
    size_t submitted = 0, issued = 0;
    auto submit = [&](size_t m) -> int {
        const size_t si = (k->stage_next++) % nstage;
        Staging &sg = k->stage[si];
        if (sg.pending) {
            const int r = (c->fault_kind == 3) ? fail(VR_ERR_TIMEOUT, "staging wait expired (injected)")
                                               : wait_event(sg.done, kWaitSeconds);
            if (r != VR_OK) return r;
            sg.pending = false;
        }
        st_of[m] = si;
        const DrawBrick brick = db[misses[m].first];
        void *dst = sg.host;
        const bool inject = c->fault_kind == 1 && k->generated == c->fault_after;
        k->generated++;
        try {
            jobs[m] = produce_brick(k->workers, cb, brick, dst, inject);
        } catch (const std::exception &e) {       // the job's buffers could not be had
            return fail(VR_ERR_OOM, e.what());
        }
        return VR_OK;
    };
    while (issued < misses.size() && rc == VR_OK) {
        while (submitted < misses.size() && submitted < issued + nstage && rc == VR_OK) rc = submit(submitted++);
        if (rc != VR_OK) break;
        const size_t m = issued;
        BrickJob &job = *jobs[m];
        if (job.finished.wait_for(std::chrono::duration<double>(kWaitSeconds)) != std::future_status::ready) {
            rc = fail(VR_ERR_TIMEOUT, "brick production did not finish within its time bound");
            break;
        }
        job.finished.get();
        if (!job.err.empty()) {
            rc = fail(VR_ERR_IO, job.err);
            break;
        }
        const int si = misses[m].second;
        Slot &s = k->slots[si];
        const DrawBrick &b = db[misses[m].first];
        Staging &sg = k->stage[st_of[m]];
        // (errors leave through the loop's end, which lets the producers still running finish)
        cudaError_t ce = s.used ? cudaStreamWaitEvent(k->copy, s.last_use, 0) : cudaSuccess;
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(k->d_base + (size_t)si * k->slot_bytes, sg.host, (size_t)b.bytes,
                                 cudaMemcpyHostToDevice, k->copy);
        if (ce == cudaSuccess) ce = cudaEventRecord(sg.done, k->copy);
        if (ce != cudaSuccess) {
            rc = cuda_fail(ce, "brick copy to the cache");
            break;
        }
        sg.pending = true;
        s.cube = cb->id;
        s.exp2 = job.exp2;
        k->where[key_of(cb->id, s.brick)] = si;
        db[misses[m].first].data_off = (long long)((size_t)si * k->slot_bytes / esz);
        db[misses[m].first].exp2 = job.exp2;
        db[misses[m].first].atlas = 0ull;
        k->misses++;
        k->bytes += b.bytes;
        ++issued;
        if (atlas) {
            if ((rc = slot_atlas_pack(c, cb, si, b, g)) != VR_OK) {
                k->where.erase(key_of(cb->id, s.brick));
                s.cube = -1;
                s.brick = -1;
                s.chunk = -1;
                break;
            }
            db[misses[m].first].atlas = s.tex;
            db[misses[m].first].alog = s.alog;
        }
    }
    if (rc != VR_OK) {
        // let submitted producers finish (they write into staging we own), drop unfilled slots
        for (size_t m = 0; m < submitted; ++m)
            if (jobs[m] && jobs[m]->finished.valid())   // (not yet taken by get())
                jobs[m]->finished.wait_for(std::chrono::duration<double>(kWaitSeconds));
        for (size_t m = issued; m < misses.size(); ++m) {
            Slot &s = k->slots[misses[m].second];
            s.cube = -1;
            s.brick = -1;
            s.chunk = -1;
        }
        return rc;
    }
    return VR_OK;
}

// Frame of a streamed cube: work-list, chunks of at most `nslots` bricks made resident and
// ray-cast, then one compositing pass.
int render_streamed(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s) {
    int rc = cache_create(c);
    if (rc) return rc;
    BrickCache *k = c->cache;
    std::lock_guard<std::recursive_mutex> lock(k->mu);
    size_t max_bytes = 0;
    for (auto &b : cb->tmpl) max_bytes = std::max(max_bytes, (size_t)b.bytes);
    if ((rc = cache_size(c, max_bytes)) != VR_OK) return rc;
    FrameConsts fc = make_consts(c, cb);
    // timing (vr_set_timing): frame, ray casting (from the first chunk's residency to the last
    // chunk's ray-cast, so it includes waits for bricks made resident during the frame) and
    // compositing
    FrameTiming tm(c);
    cudaEvent_t *ev = tm.ev;
    if (c->timing && (rc = timing_events(c, ev)) != VR_OK) return rc;
    WorkList wl;
    build_worklist(c, cb, wl);
    const size_t nd = wl.db.size();
    // chunks of whole bricks (their items are contiguous in the work-list)
    std::vector<size_t> item_start(nd + 1, 0);
    for (auto &it : wl.items) item_start[it.db + 1]++;
    for (size_t i = 0; i < nd; ++i) item_start[i + 1] += item_start[i];
    const size_t per = (size_t)k->nslots;
    const size_t nchunks = nd == 0 ? 0 : (nd + per - 1) / per;
    // staged upload: table, all bricks (composite), bins, then per chunk its bricks and items
    size_t off = 0;
    wl.off_lut = off; off = align_up(off + sizeof(float4) * c->lut.size(), 256);
    wl.off_db = off; off = align_up(off + sizeof(DrawBrick) * nd, 256);
    wl.off_ts = off; off = align_up(off + sizeof(int) * wl.tile_start.size(), 256);
    wl.off_tl = off; off = align_up(off + sizeof(int) * wl.tile_list.size(), 256);
    wl.off_mask = off; off = align_up(off + c->chmask.size(), 256);
    std::vector<size_t> off_cdb(nchunks), off_cit(nchunks);
    for (size_t ch = 0; ch < nchunks; ++ch) {
        const size_t d0 = ch * per, d1 = std::min(nd, d0 + per);
        off_cdb[ch] = off; off = align_up(off + sizeof(DrawBrick) * (d1 - d0), 256);
        off_cit[ch] = off; off = align_up(off + sizeof(TileItem) * (item_start[d1] - item_start[d0]), 256);
    }
    wl.bytes = off;
    if (c->frame_pending) {
        CK(cudaEventSynchronize(c->upload_done));
        CK(cudaStreamWaitEvent(s, c->frame_done, 0));
    }
    if ((rc = ensure_host(c, wl.bytes)) != VR_OK) return rc;
    if ((rc = ensure(c->d_stage, wl.bytes, c)) != VR_OK) return rc;
    if (ev[0]) CK(cudaEventRecord(ev[0], s));
    const size_t felem = c->mode == VR_DVR ? sizeof(float4) : sizeof(float);
    c->frag_valid = false;             // d_frags now holds this streamed frame's fragments
    if ((rc = ensure(c->d_frags, std::max<size_t>((size_t)wl.frag_px * felem, 16), c)) != VR_OK) return rc;
    const size_t opix = (size_t)fc.cam.W * fc.cam.H, ofl = opix * (c->mode == VR_DVR ? 4 : 1);
    const bool direct = out_where == VR_DEVICE && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
    float *dst = out;
    if (!direct) {
        if ((rc = ensure(c->d_out, ofl, c)) != VR_OK) return rc;
        dst = c->d_out.p;
    }
    char *h = c->h_stage, *d = c->d_stage.p;
    std::memcpy(h + wl.off_lut, c->lut.data(), sizeof(float4) * c->lut.size());
    std::memcpy(h + wl.off_ts, wl.tile_start.data(), sizeof(int) * wl.tile_start.size());
    if (!wl.tile_list.empty()) std::memcpy(h + wl.off_tl, wl.tile_list.data(), sizeof(int) * wl.tile_list.size());
    if (!c->chmask.empty()) std::memcpy(h + wl.off_mask, c->chmask.data(), c->chmask.size());
    // the shared part (table, bins, mask) first; brick records once every chunk is resident
    CK(cudaMemcpyAsync(d, h, wl.off_db, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d + wl.off_ts, h + wl.off_ts, wl.off_mask - wl.off_ts + c->chmask.size(),
                       cudaMemcpyHostToDevice, s));
    if (!c->chmask.empty()) fc.chmask = reinterpret_cast<const unsigned char *>(d + wl.off_mask);
    if (ev[1]) CK(cudaEventRecord(ev[1], s));
    for (size_t ch = 0; ch < nchunks; ++ch) {
        const size_t d0 = ch * per, d1 = std::min(nd, d0 + per);
        const int64_t chunk_id = ++k->chunk_counter;
        if ((rc = make_resident(c, cb, wl.db, d0, d1, chunk_id)) != VR_OK) {
            // leave nothing in flight that reads the staging of this abandoned frame
            cudaStreamSynchronize(k->copy);
            cudaStreamSynchronize(s);
            return rc;
        }
        CK(cudaEventRecord(k->copies_done, k->copy));
        CK(cudaStreamWaitEvent(s, k->copies_done, 0));
        DrawBrick *hdb = reinterpret_cast<DrawBrick *>(h + off_cdb[ch]);
        for (size_t i = d0; i < d1; ++i) hdb[i - d0] = wl.db[i];
        TileItem *hit = reinterpret_cast<TileItem *>(h + off_cit[ch]);
        const size_t i0 = item_start[d0], i1 = item_start[d1];
        for (size_t i = i0; i < i1; ++i) {
            hit[i - i0] = wl.items[i];
            hit[i - i0].db -= (int)d0;
        }
        CK(cudaMemcpyAsync(d + off_cdb[ch], h + off_cdb[ch], off_cit[ch] - off_cdb[ch] + sizeof(TileItem) * (i1 - i0),
                           cudaMemcpyHostToDevice, s));
        CK(launch_raycast(fc, reinterpret_cast<const float4 *>(d + wl.off_lut),
                          reinterpret_cast<const DrawBrick *>(d + off_cdb[ch]),
                          reinterpret_cast<const TileItem *>(d + off_cit[ch]), (int)(i1 - i0), k->d_base,
                          c->d_frags.p, c->d_ctr, s));
        for (size_t i = d0; i < d1; ++i) {
            Slot &sl = k->slots[k->where[key_of(cb->id, wl.db[i].brick)]];
            // one event stands for every reader: frames of other streams may still read this
            // slot, so the new record first waits for the previous one (which was enqueued
            // earlier: no cycle); an eviction waiting on it then waits for all of them
            if (sl.used) CK(cudaStreamWaitEvent(s, sl.last_use, 0));
            CK(cudaEventRecord(sl.last_use, s));
            sl.used = true;
        }
    }
    if (ev[2]) CK(cudaEventRecord(ev[2], s));
    std::memcpy(h + wl.off_db, wl.db.data(), sizeof(DrawBrick) * nd);
    CK(cudaMemcpyAsync(d + wl.off_db, h + wl.off_db, sizeof(DrawBrick) * nd, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->upload_done, s));
    CK(launch_composite(fc, reinterpret_cast<const DrawBrick *>(d + wl.off_db),
                        reinterpret_cast<const int *>(d + wl.off_ts), reinterpret_cast<const int *>(d + wl.off_tl),
                        c->d_frags.p, dst, s));
    if (ev[3]) CK(cudaEventRecord(ev[3], s));
    if (!direct)
        CK(cudaMemcpyAsync(out, dst, ofl * sizeof(float),
                           out_where == VR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(c->frame_done, s));
    c->frame_pending = true;
    tm.queue();
    c->frames++;
    c->fragments += wl.frag_px;
    c->bricks_drawn += (int64_t)nd;
    if (out_where == VR_HOST && !c->async_host_out) CK(cudaStreamSynchronize(s));
    return VR_OK;
}

// DVR frame of a streamed or compressed cube with global early termination: the frame's bricks
// (the work-list: visible, not skipped) are made resident together, then one ray-march launch
// walks the whole brick grid as for a resident cube.  Bricks outside the work-list are walked
// through without samples: no ray of the frame reaches them (their screen rectangle misses
// the frame) or their values map to zero opacity, exactly as the fragment path leaves them out.
int render_streamed_global(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s) {
    int rc = cache_create(c);
    if (rc) return rc;
    BrickCache *k = c->cache;
    std::lock_guard<std::recursive_mutex> lock(k->mu);
    size_t max_bytes = 0;
    for (auto &b : cb->tmpl) max_bytes = std::max(max_bytes, (size_t)b.bytes);
    if ((rc = cache_size(c, max_bytes)) != VR_OK) return rc;
    FrameConsts fc = make_consts(c, cb);
    WorkList wl;
    build_worklist(c, cb, wl);
    const size_t nd = wl.db.size(), nb = cb->tmpl.size();
    if (nd > (size_t)k->nslots)
        return fail(VR_ERR_UNSUPPORTED, "global termination needs every brick of the frame in the brick cache at once");
    FrameTiming tm(c);
    cudaEvent_t *ev = tm.ev;
    if (c->timing && (rc = timing_events(c, ev)) != VR_OK) return rc;
    size_t off = 0;
    const size_t off_lut = off;
    off = align_up(off + sizeof(float4) * c->lut.size(), 256);
    const size_t off_b = off;
    off = align_up(off + sizeof(DrawBrick) * nb, 256);
    const size_t off_mask = off;
    off = align_up(off + c->chmask.size(), 256);
    if (c->frame_pending) {
        CK(cudaEventSynchronize(c->upload_done));
        CK(cudaStreamWaitEvent(s, c->frame_done, 0));
    }
    if ((rc = ensure_host(c, off)) != VR_OK) return rc;
    if ((rc = ensure(c->d_stage, off, c)) != VR_OK) return rc;
    if (ev[0]) CK(cudaEventRecord(ev[0], s));
    const int64_t chunk_id = ++k->chunk_counter;
    if ((rc = make_resident(c, cb, wl.db, 0, nd, chunk_id)) != VR_OK) {
        cudaStreamSynchronize(k->copy);
        if (ev[0]) cudaStreamSynchronize(s);   // its timing events go back to the pool
        return rc;
    }
    CK(cudaEventRecord(k->copies_done, k->copy));
    CK(cudaStreamWaitEvent(s, k->copies_done, 0));
    char *h = c->h_stage, *d = c->d_stage.p;
    std::memcpy(h + off_lut, c->lut.data(), sizeof(float4) * c->lut.size());
    DrawBrick *hb = reinterpret_cast<DrawBrick *>(h + off_b);
    for (size_t i = 0; i < nb; ++i) {
        hb[i] = cb->tmpl[i];
        hb[i].skip = 1;
        hb[i].sampled = 0;
        hb[i].atlas = 0ull;
    }
    for (size_t i = 0; i < nd; ++i) {
        DrawBrick b = wl.db[i];
        b.skip = 0;
        b.sampled = 0;
        hb[b.brick] = b;
    }
    if (!c->chmask.empty()) std::memcpy(h + off_mask, c->chmask.data(), c->chmask.size());
    const MarchGrid g = march_grid(c, cb);
    CK(cudaMemcpyAsync(d, h, off, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->upload_done, s));
    if (!c->chmask.empty()) fc.chmask = reinterpret_cast<const unsigned char *>(d + off_mask);
    const size_t opix = (size_t)fc.cam.W * fc.cam.H;
    float *dst = out;
    const bool direct = out_where == VR_DEVICE && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
    if (!direct) {
        if ((rc = ensure(c->d_out, opix * 4, c)) != VR_OK) return rc;
        dst = c->d_out.p;
    }
    if (ev[1]) CK(cudaEventRecord(ev[1], s));
    const bool empty = g.chi[0] <= g.clo[0] || g.chi[1] <= g.clo[1] || g.chi[2] <= g.clo[2];
    if (empty || nd == 0) {            // nothing to sample: a transparent frame
        CK(cudaMemsetAsync(dst, 0, opix * sizeof(float4), s));
    } else {
        CK(launch_raymarch(fc, reinterpret_cast<const float4 *>(d + off_lut), reinterpret_cast<DrawBrick *>(d + off_b),
                           g, k->d_base, reinterpret_cast<float4 *>(dst), c->d_ctr, s));
    }
    for (size_t i = 0; i < nd; ++i) {  // every slot this frame read: its readers' event
        Slot &sl = k->slots[k->where[key_of(cb->id, wl.db[i].brick)]];
        if (sl.used) CK(cudaStreamWaitEvent(s, sl.last_use, 0));
        CK(cudaEventRecord(sl.last_use, s));
        sl.used = true;
    }
    if (ev[2]) CK(cudaEventRecord(ev[2], s));
    if (ev[3]) CK(cudaEventRecord(ev[3], s));
    if (!direct)
        CK(cudaMemcpyAsync(out, dst, opix * sizeof(float4),
                           out_where == VR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(c->frame_done, s));
    c->frame_pending = true;
    tm.queue();
    c->frames++;
    c->bricks_drawn += (int64_t)nd;
    if (out_where == VR_HOST && !c->async_host_out) CK(cudaStreamSynchronize(s));
    return VR_OK;
}

// Set-up for a streamed or compressed cube whose cache slots keep slice atlases: sizes the cache
// for its bricks and gives as many slots as it has bricks (at most all slots) an atlas array, so
// that frames only pack.  Arrays already fit for its bricks are kept.
int cache_prepare_atlases(vr_ctx *c, Cube *cb) {
    int rc = cache_create(c);
    if (rc) return rc;
    BrickCache *k = c->cache;
    std::lock_guard<std::recursive_mutex> lock(k->mu);
    size_t max_bytes = 0;
    for (auto &b : cb->tmpl) max_bytes = std::max(max_bytes, (size_t)b.bytes);
    if ((rc = cache_size(c, max_bytes)) != VR_OK) return rc;
    SlotAtlasGeom g;
    if ((rc = slot_atlas_geom(c, cb, g)) != VR_OK) return rc;
    const int n = (int)std::min<size_t>((size_t)k->nslots, cb->tmpl.size());
    for (int i = 0; i < n; ++i)
        if ((rc = slot_atlas_alloc(c, cb, i, g)) != VR_OK) return rc;
    return VR_OK;
}

// Brick `brick` of a streamed cube as stored (generated on the calling thread; compressed
// cubes: decoded on the device and copied back).
int streamed_brick(Cube *cb, int64_t brick, void *data, int *exp2) {
    const DrawBrick &b = cb->tmpl[brick];
    int e = 0;
    if (cb->wavelet) {
        float *tmp = nullptr;
        CK(cudaMalloc(&tmp, (size_t)b.bytes));
        cudaError_t er = launch_wavelet_decode(cb->d_wstore, (int)cb->n[0], (int)cb->n[1], (int)cb->n[2], b.org,
                                               b.dim, tmp, 0);
        if (er == cudaSuccess) er = cudaMemcpy(data, tmp, (size_t)b.bytes, cudaMemcpyDeviceToHost);
        cudaFree(tmp);
        if (er != cudaSuccess) return cuda_fail(er, "wavelet brick decode");
        *exp2 = 0;
        return VR_OK;
    }
    if (cb->storage == VR_F32) {
        gen_region(cb->proc_seed, cb->n, b.org, b.dim, static_cast<float *>(data));
    } else {
        const size_t count = (size_t)b.dim[0] * b.dim[1] * b.dim[2];
        std::vector<float> tmp(count);
        gen_region(cb->proc_seed, cb->n, b.org, b.dim, tmp.data());
        e = encode_region(tmp.data(), count, cb->storage, data);
    }
    *exp2 = e;
    return VR_OK;
}

int streamed_exp(Cube *cb, int64_t brick, int *exp2) {
    if (cb->storage == VR_F32) {
        *exp2 = 0;
        return VR_OK;
    }
    const DrawBrick &b = cb->tmpl[brick];
    const size_t count = (size_t)b.dim[0] * b.dim[1] * b.dim[2];
    std::vector<uint16_t> codes(count);
    return streamed_brick(cb, brick, codes.data(), exp2);
}

}  // namespace vrh
