// vr_serve.cu -- an interactive request loop with continuous batching.
//
// The paper's server waits for render requests carrying the viewer's matrices and colour map
// and answers each with a frame (Section 2.3).  Here many such requests arrive over time for
// several cubes at different resolutions; every request that has arrived is admitted as soon as
// a frame slot (a CUDA stream with its own scratch) is free and, for streamed cubes, the brick
// cache has room for the bricks it still needs without evicting bricks of frames in flight.
// Admitted frames run concurrently on their slots' streams; each completes on its own event,
// and its latency is measured from its arrival to the completion seen by the loop.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <future>
#include <thread>
#include <vector>

#include "vr_host.h"

namespace vrh {
namespace {

struct FrameSlot {
    vr_ctx *c = nullptr;              // frame context sharing the parent's cubes, counters, cache
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    int req = -1;                     // request in flight, -1 = free
    Cube *cube = nullptr;
    std::vector<int64_t> held;        // streamed bricks this frame holds in the cache
    bool loading = false;             // streamed frame: bricks still being made resident
    std::future<int> load;            // ... by a host thread that then queues the frame
    std::vector<int64_t> bricks;      // its bricks, held once the frame is queued
};

// A frame context: own stream state and scratch, shared cubes / counters / brick cache.
vr_ctx *slot_context(vr_ctx *parent) {
    vr_ctx *c = new vr_ctx();
    c->device = parent->device;
    c->cubes = parent->cubes;
    c->next_id = -1;
    c->d_ctr = parent->d_ctr;
    c->cache = parent->cache;
    c->cache_bytes = parent->cache_bytes;
    c->async_host_out = true;          // completion is the slot's event, not a host sync
    c->fault_kind = parent->fault_kind;
    c->fault_after = parent->fault_after;
    return c;
}

void slot_release(vr_ctx *c) {
    if (!c) return;
    if (c->frame_pending) cudaEventSynchronize(c->frame_done);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->d_stage.p) cudaFree(c->d_stage.p);
    if (c->d_frags.p) cudaFree(c->d_frags.p);
    if (c->d_out.p) cudaFree(c->d_out.p);
    if (c->upload_done) cudaEventDestroy(c->upload_done);
    if (c->frame_done) cudaEventDestroy(c->frame_done);
    delete c;                          // cubes, counters and cache belong to the parent
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace vrh

using namespace vrh;

#pragma GCC visibility push(default)
extern "C" int vr_serve(vr_ctx *c, const vr_request *reqs, int n, const vr_serve_config *cfg,
                        vr_request_result *res, vr_serve_summary *sum) {
    if (!c || (!reqs && n > 0) || !cfg || (!res && n > 0)) return arg_fail("null argument");
    if (n < 0 || cfg->max_inflight < 1 || cfg->max_inflight > 64) return arg_fail("max_inflight must be 1..64");
    for (int i = 0; i < n; ++i) {
        if (!reqs[i].out || !reqs[i].lut || reqs[i].nlut < 2) return arg_fail("request without output or table");
        if (!find_cube(c, reqs[i].cube_id)) return VR_ERR_NOT_FOUND;
        if (i > 0 && reqs[i].arrival_ms < reqs[i - 1].arrival_ms) return arg_fail("requests must be in arrival order");
    }
    int rc = set_dev(c);
    if (rc) return rc;
    bool any_streamed = false;
    for (int i = 0; i < n; ++i) any_streamed |= find_cube(c, reqs[i].cube_id)->streamed;
    if (any_streamed && (rc = cache_create(c)) != VR_OK) return rc;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    // frame slots
    std::vector<FrameSlot> slots(cfg->max_inflight);
    auto cleanup = [&]() {
        for (auto &sl : slots) {
            if (sl.loading && sl.load.valid()) sl.load.wait();
            if (sl.s) cudaStreamSynchronize(sl.s);
            if (sl.c) {
                c->frames += sl.c->frames;
                c->fragments += sl.c->fragments;
                c->bricks_drawn += sl.c->bricks_drawn;
                if (sl.cube && !sl.held.empty()) cache_hold(c, sl.cube, sl.held, -1, true);
            }
            slot_release(sl.c);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.s) cudaStreamDestroy(sl.s);
        }
    };
    for (auto &sl : slots) {
        sl.c = slot_context(c);
        if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.c->upload_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.c->frame_done, cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return fail(VR_ERR_CUDA, "could not create the frame slots' streams and events");
        }
    }
    for (int i = 0; i < n; ++i) {
        res[i] = vr_request_result{};
        res[i].status = VR_ERR_STATE;
    }
    std::deque<int> queue;             // arrived, not yet admitted (arrival order)
    std::vector<double> lat;
    lat.reserve(n);
    // brick holds (+1 when a streamed frame is queued, -1 when it completes), applied in order
    // whenever the cache lock is free: they only steer admission, never correctness
    struct HoldOp {
        Cube *cube;
        std::vector<int64_t> bricks;
        int delta;
    };
    std::deque<HoldOp> holds;
    int next = 0, finished = 0, inflight = 0, max_conc = 0;
    int64_t failed = 0;
    const auto t0 = std::chrono::steady_clock::now();
    auto finish = [&](int ri, int status) {
        vr_request_result &r = res[ri];
        r.done_ms = ms_since(t0);
        r.latency_ms = r.done_ms - reqs[ri].arrival_ms;
        r.status = status;
        if (status == VR_OK) lat.push_back(r.latency_ms); else ++failed;
        ++finished;
    };
    while (finished < n) {
        const double now = ms_since(t0);
        while (next < n && reqs[next].arrival_ms <= now) queue.push_back(next++);
        bool progress = false;
        while (!holds.empty() && cache_hold(c, holds.front().cube, holds.front().bricks, holds.front().delta, false))
            holds.pop_front();
        // streamed frames whose bricks are resident and whose kernels are now queued
        for (auto &sl : slots) {
            if (sl.req < 0 || !sl.loading) continue;
            if (sl.load.wait_for(std::chrono::seconds(0)) != std::future_status::ready) continue;
            const int st = sl.load.get();
            sl.loading = false;
            progress = true;
            if (st != VR_OK) {
                finish(sl.req, st);
                --inflight;
                sl.req = -1;
                continue;
            }
            sl.held = std::move(sl.bricks);
            sl.bricks.clear();
            holds.push_back({sl.cube, sl.held, +1});
        }
        // completions
        for (auto &sl : slots) {
            if (sl.req < 0 || sl.loading) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            finish(sl.req, q == cudaSuccess ? VR_OK : cuda_fail(q, "frame completion"));
            if (sl.cube && !sl.held.empty()) holds.push_back({sl.cube, std::move(sl.held), -1});
            sl.held.clear();
            sl.req = -1;
            --inflight;
            progress = true;
        }
        // admissions, in arrival order, while frame slots last; a streamed request whose
        // bricks cannot be made room for now (or whose cache is busy) lets later ones pass
        for (size_t qi = 0; qi < queue.size();) {
            FrameSlot *free_slot = nullptr;
            for (auto &sl : slots)
                if (sl.req < 0) { free_slot = &sl; break; }
            if (!free_slot) break;
            const int ri = queue[qi];
            const vr_request &q = reqs[ri];
            vr_ctx *fc = free_slot->c;
            Cube *cb = find_cube(c, q.cube_id);
            int st = vr_set_transfer_function(fc, q.lut, q.nlut, q.vmin, q.vmax);
            if (st == VR_OK) st = vr_set_camera(fc, q.view, q.proj, q.param, q.width, q.height);
            if (st == VR_OK) st = vr_set_render_params(fc, q.mode, q.step, q.ert_threshold);
            if (st == VR_OK) st = vr_set_termination(fc, q.termination);
            if (st == VR_OK) st = check_ready(fc, cb);
            std::vector<int64_t> bricks;
            if (st == VR_OK && cb->streamed) {
                WorkList wl;
                build_worklist(fc, cb, wl);
                int64_t missing = 0, free_slots = 0;
                const int m = cache_missing(c, cb, wl, &missing, &free_slots);
                // wait while the cache is busy or the bricks the request lacks would displace
                // bricks of frames in flight (one larger than the whole cache runs alone)
                if (m == VR_ERR_TIMEOUT || (m == VR_OK && missing > free_slots && inflight > 0)) {
                    ++qi;
                    continue;
                }
                st = m;
                for (auto &d : wl.db) bricks.push_back(d.brick);
            }
            queue.erase(queue.begin() + qi);
            res[ri].admit_ms = ms_since(t0);
            progress = true;
            if (st == VR_OK && cb->streamed) {
                // bricks are produced and copied from a host thread; the loop keeps serving
                FrameSlot *sl = free_slot;
                const int dev = c->device;
                sl->load = std::async(std::launch::async, [sl, fc, cb, &q, dev]() {
                    if (cudaSetDevice(dev) != cudaSuccess) return (int)VR_ERR_CUDA;
                    int r = render_frame_impl(fc, cb, q.out, q.out_where, sl->s);
                    if (r == VR_OK && cudaEventRecord(sl->done, sl->s) != cudaSuccess) r = VR_ERR_CUDA;
                    return r;
                });
                sl->loading = true;
                sl->bricks = std::move(bricks);
                sl->req = ri;
                sl->cube = cb;
                ++inflight;
                max_conc = std::max(max_conc, inflight);
                continue;
            }
            if (st == VR_OK) st = render_frame_impl(fc, cb, q.out, q.out_where, free_slot->s);
            if (st == VR_OK) st = cudaEventRecord(free_slot->done, free_slot->s) == cudaSuccess ? VR_OK : VR_ERR_CUDA;
            if (st != VR_OK) {
                finish(ri, st);
                continue;
            }
            free_slot->req = ri;
            free_slot->cube = cb;
            ++inflight;
            max_conc = std::max(max_conc, inflight);
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (auto &h : holds) cache_hold(c, h.cube, h.bricks, h.delta, true);
    const double wall = ms_since(t0);
    cleanup();
    if (sum) {
        std::memset(sum, 0, sizeof(*sum));
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) {
            if (lat.empty()) return 0.0;
            const size_t i = std::min(lat.size() - 1, (size_t)std::ceil(p * lat.size()) - (p > 0 ? 1 : 0));
            return lat[i];
        };
        sum->completed = (int64_t)lat.size();
        sum->failed = failed;
        sum->wall_ms = wall;
        sum->p50_ms = pct(0.50);
        sum->p99_ms = pct(0.99);
        sum->max_ms = lat.empty() ? 0.0 : lat.back();
        sum->frames_per_s = wall > 0 ? 1e3 * (double)lat.size() / wall : 0.0;
        sum->max_concurrent = max_conc;
    }
    return failed ? VR_ERR_STATE : VR_OK;
}
#pragma GCC visibility pop
