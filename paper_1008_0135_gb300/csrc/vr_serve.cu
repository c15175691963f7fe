// vr_serve.cu -- an interactive request loop with continuous batching.
//
// The paper's server waits for render requests carrying the viewer's matrices and colour map
// and answers each with a frame (Section 2.3).  Here many such requests arrive over time for
// several cubes at different resolutions; every request that has arrived is admitted as soon as
// a frame slot (a CUDA stream with its own scratch) is free and, for streamed cubes, the brick
// cache has room for the bricks it still needs without evicting bricks of frames in flight.
// Admitted frames run concurrently on their slots' streams; each completes on its own event,
// and its latency is measured from its arrival to the completion seen by the loop.
//
// One loop (ServeCore) serves two front ends: vr_serve replays a trace of requests with known
// arrival times and returns when all are done; the online server (vr_serve_open / submit /
// poll / close) runs the loop on a host thread of its own while the caller submits requests
// whenever they arrive and collects the finished ones.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <future>
#include <memory>
#include <new>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vr_host.h"

namespace vrh {
namespace {

// One request as the loop keeps it: a copy of the caller's request with its own table.
struct Req {
    vr_request q{};
    std::vector<float> lut;
    double arrival_ms = 0.0;          // ms after the loop started
    vr_request_result res{};
    int64_t ticket = -1;
};

struct FrameSlot {
    vr_ctx *c = nullptr;              // frame context sharing the parent's cubes, counters, cache
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    Req *req = nullptr;               // request in flight, nullptr = free
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

// Copies a request (and its table) for the loop; checks what can be checked before admission.
int make_req(vr_ctx *c, const vr_request &src, Req &r) {
    if (!src.out || !src.lut || src.nlut < 2 || src.nlut > kMaxLut) return arg_fail("request without output or table");
    if (!find_cube(c, src.cube_id)) return VR_ERR_NOT_FOUND;
    r.q = src;
    r.lut.assign(src.lut, src.lut + (size_t)4 * src.nlut);
    r.q.lut = r.lut.data();
    r.res = vr_request_result{};
    r.res.status = VR_ERR_STATE;
    return VR_OK;
}

// The continuous-batching loop.  Single-threaded: only the thread that calls step() touches it.
struct ServeCore {
    vr_ctx *c = nullptr;
    std::vector<FrameSlot> slots;
    std::deque<Req *> queue;           // arrived, not yet admitted (arrival order)
    // brick holds (+1 when a streamed frame is queued, -1 when it completes), applied in order
    // whenever the cache lock is free: they only steer admission, never correctness
    struct HoldOp {
        Cube *cube;
        std::vector<int64_t> bricks;
        int delta;
    };
    std::deque<HoldOp> holds;
    std::vector<double> lat;
    std::vector<Req *> finished;       // completed or failed since the caller last took them
    int inflight = 0, max_conc = 0;
    int64_t failed = 0, done = 0;
    std::chrono::steady_clock::time_point t0;

    int open(vr_ctx *parent, int max_inflight) {
        c = parent;
        t0 = std::chrono::steady_clock::now();
        slots.resize(max_inflight);
        for (auto &sl : slots) {
            sl.c = slot_context(c);
            if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.c->upload_done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.c->frame_done, cudaEventDisableTiming) != cudaSuccess)
                return fail(VR_ERR_CUDA, "could not create the frame slots' streams and events");
        }
        return VR_OK;
    }

    // Waits for every slot, returns the slots' statistics to the parent, releases the slots.
    void close() {
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
        for (auto &h : holds) cache_hold(c, h.cube, h.bricks, h.delta, true);
        holds.clear();
        slots.clear();
    }

    double now() const { return ms_since(t0); }

    // After a host-side exception in the loop: waits for the frames in flight (their streams and
    // brick loads), then fails every request the loop still holds, queued or in a slot.
    void abandon() {
        for (auto &sl : slots) {
            if (sl.loading && sl.load.valid()) sl.load.wait();
            sl.loading = false;
            if (sl.s) cudaStreamSynchronize(sl.s);
            if (sl.req) {
                Req *r = sl.req;
                sl.req = nullptr;
                --inflight;
                finish(r, VR_ERR_STATE);
            }
        }
        while (!queue.empty()) {
            finish(queue.front(), VR_ERR_STATE);
            queue.pop_front();
        }
    }

    void finish(Req *r, int status) {
        r->res.done_ms = now();
        r->res.latency_ms = r->res.done_ms - r->arrival_ms;
        r->res.status = status;
        if (status == VR_OK) lat.push_back(r->res.latency_ms); else ++failed;
        ++done;
        finished.push_back(r);
    }

    bool idle() const { return queue.empty() && inflight == 0; }

    // One pass: cache holds, streamed frames now queued, completions, admissions.
    bool step() {
        bool progress = false;
        while (!holds.empty() && cache_hold(c, holds.front().cube, holds.front().bricks, holds.front().delta, false))
            holds.pop_front();
        // streamed frames whose bricks are resident and whose kernels are now queued
        for (auto &sl : slots) {
            if (!sl.req || !sl.loading) continue;
            if (sl.load.wait_for(std::chrono::seconds(0)) != std::future_status::ready) continue;
            const int st = sl.load.get();
            sl.loading = false;
            progress = true;
            if (st != VR_OK) {
                finish(sl.req, st);
                --inflight;
                sl.req = nullptr;
                continue;
            }
            sl.held = std::move(sl.bricks);
            sl.bricks.clear();
            holds.push_back({sl.cube, sl.held, +1});
        }
        // completions
        for (auto &sl : slots) {
            if (!sl.req || sl.loading) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            finish(sl.req, q == cudaSuccess ? VR_OK : cuda_fail(q, "frame completion"));
            if (sl.cube && !sl.held.empty()) holds.push_back({sl.cube, std::move(sl.held), -1});
            sl.held.clear();
            sl.req = nullptr;
            --inflight;
            progress = true;
        }
        // admissions, in arrival order, while frame slots last; a streamed request whose
        // bricks cannot be made room for now (or whose cache is busy) lets later ones pass
        for (size_t qi = 0; qi < queue.size();) {
            FrameSlot *free_slot = nullptr;
            for (auto &sl : slots)
                if (!sl.req) { free_slot = &sl; break; }
            if (!free_slot) break;
            Req *r = queue[qi];
            const vr_request &q = r->q;
            vr_ctx *fc = free_slot->c;
            Cube *cb = find_cube(c, q.cube_id);
            int st = cb ? VR_OK : VR_ERR_NOT_FOUND;
            if (st == VR_OK) st = vr_set_transfer_function(fc, q.lut, q.nlut, q.vmin, q.vmax);
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
            r->res.admit_ms = now();
            progress = true;
            if (st == VR_OK && cb->streamed) {
                // bricks are produced and copied from a host thread; the loop keeps serving
                FrameSlot *sl = free_slot;
                const int dev = c->device;
                sl->load = std::async(std::launch::async, [sl, fc, cb, r, dev]() {
                    if (cudaSetDevice(dev) != cudaSuccess) return (int)VR_ERR_CUDA;
                    int rr = render_frame_impl(fc, cb, r->q.out, r->q.out_where, sl->s);
                    if (rr == VR_OK && cudaEventRecord(sl->done, sl->s) != cudaSuccess) rr = VR_ERR_CUDA;
                    return rr;
                });
                sl->loading = true;
                sl->bricks = std::move(bricks);
                sl->req = r;
                sl->cube = cb;
                ++inflight;
                max_conc = std::max(max_conc, inflight);
                continue;
            }
            if (st == VR_OK) st = render_frame_impl(fc, cb, q.out, q.out_where, free_slot->s);
            if (st == VR_OK) st = cudaEventRecord(free_slot->done, free_slot->s) == cudaSuccess ? VR_OK : VR_ERR_CUDA;
            if (st != VR_OK) {
                finish(r, st);
                continue;
            }
            free_slot->req = r;
            free_slot->cube = cb;
            ++inflight;
            max_conc = std::max(max_conc, inflight);
        }
        return progress;
    }

    void summary(vr_serve_summary *sum, double wall) {
        if (!sum) return;
        std::memset(sum, 0, sizeof(*sum));
        std::vector<double> l = lat;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            if (l.empty()) return 0.0;
            const size_t i = std::min(l.size() - 1, (size_t)std::ceil(p * l.size()) - (p > 0 ? 1 : 0));
            return l[i];
        };
        sum->completed = (int64_t)l.size();
        sum->failed = failed;
        sum->wall_ms = wall;
        sum->p50_ms = pct(0.50);
        sum->p99_ms = pct(0.99);
        sum->max_ms = l.empty() ? 0.0 : l.back();
        sum->frames_per_s = wall > 0 ? 1e3 * (double)l.size() / wall : 0.0;
        sum->max_concurrent = max_conc;
    }
};

int serve_prepare(vr_ctx *c, bool any_streamed) {
    int rc = set_dev(c);
    if (rc) return rc;
    if (any_streamed && (rc = cache_create(c)) != VR_OK) return rc;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    return VR_OK;
}

}  // namespace
}  // namespace vrh

using namespace vrh;

// The online server: the loop on its own host thread, fed by vr_serve_submit.
struct vr_server {
    vr_ctx *c = nullptr;
    ServeCore core;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;          // signals finished requests and closing
    std::unordered_map<int64_t, std::unique_ptr<Req>> owned;
    std::deque<Req *> submitted;         // not yet handed to the loop
    std::deque<Req *> completed;         // finished, not yet polled
    int64_t next_ticket = 0;
    int64_t outstanding = 0;             // submitted, not yet finished
    bool closing = false;
    bool broken = false;                 // the loop stopped on a host-side exception
    std::string broken_what;

    void run() {
        cudaSetDevice(c->device);
        try {
            loop();
        } catch (const std::exception &e) {
            stop_after_error(e.what());
        } catch (...) {
            stop_after_error("unexpected host-side exception");
        }
    }

    // The loop cannot go on: every request it holds or has not yet taken fails, waiters wake,
    // and later submissions are refused.
    void stop_after_error(const char *what) {
        try {
            core.abandon();
        } catch (...) {
        }
        std::lock_guard<std::mutex> l(mu);
        broken = true;
        try {
            broken_what = what;
            while (!submitted.empty()) {
                core.finish(submitted.front(), VR_ERR_STATE);
                submitted.pop_front();
            }
            for (Req *r : core.finished) completed.push_back(r);
        } catch (...) {
        }
        core.finished.clear();
        outstanding = 0;
        cv.notify_all();
    }

    void loop() {
        for (;;) {
            {
                std::lock_guard<std::mutex> l(mu);
                while (!submitted.empty()) {
                    core.queue.push_back(submitted.front());
                    submitted.pop_front();
                }
            }
            const bool progress = core.step();
            bool stop = false;
            {
                std::lock_guard<std::mutex> l(mu);
                if (!core.finished.empty()) {
                    for (Req *r : core.finished) completed.push_back(r);
                    outstanding -= (int64_t)core.finished.size();
                    core.finished.clear();
                    cv.notify_all();
                }
                stop = closing && outstanding == 0 && submitted.empty() && core.idle();
            }
            if (stop) break;
            if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
};

#pragma GCC visibility push(default)
static int vr_serve_body(vr_ctx *c, const vr_request *reqs, int n, const vr_serve_config *cfg,
                        vr_request_result *res, vr_serve_summary *sum);
extern "C" int vr_serve(vr_ctx *c, const vr_request *reqs, int n, const vr_serve_config *cfg,
                        vr_request_result *res, vr_serve_summary *sum) {
    return abi_guard([&] { return vr_serve_body(c, reqs, n, cfg, res, sum); });
}
static int vr_serve_body(vr_ctx *c, const vr_request *reqs, int n, const vr_serve_config *cfg,
                        vr_request_result *res, vr_serve_summary *sum) {
    if (!c || (!reqs && n > 0) || !cfg || (!res && n > 0)) return arg_fail("null argument");
    if (n < 0 || cfg->max_inflight < 1 || cfg->max_inflight > 64) return arg_fail("max_inflight must be 1..64");
    std::vector<Req> rq;
    try {
        rq.resize(n);
    } catch (const std::bad_alloc &) {
        return fail(VR_ERR_OOM, "no host memory for the requests");
    }
    bool any_streamed = false;
    for (int i = 0; i < n; ++i) {
        const int rc = make_req(c, reqs[i], rq[i]);
        if (rc != VR_OK) return rc;
        if (i > 0 && reqs[i].arrival_ms < reqs[i - 1].arrival_ms) return arg_fail("requests must be in arrival order");
        rq[i].arrival_ms = reqs[i].arrival_ms;
        any_streamed |= find_cube(c, reqs[i].cube_id)->streamed;
    }
    int rc = serve_prepare(c, any_streamed);
    if (rc) return rc;
    ServeCore core;
    if ((rc = core.open(c, cfg->max_inflight)) != VR_OK) {
        core.close();
        return rc;
    }
    int next = 0;
    try {
        while (core.done < n) {
            const double now = core.now();
            while (next < n && rq[next].arrival_ms <= now) core.queue.push_back(&rq[next++]);
            const bool progress = core.step();
            core.finished.clear();
            if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    } catch (const std::exception &e) {
        // no frame of this call may still write into the callers' outputs after it returns
        rc = fail(VR_ERR_STATE, e.what());
        core.abandon();
        for (int i = next; i < n; ++i) core.finish(&rq[i], VR_ERR_STATE);
    }
    const double wall = core.now();
    core.close();
    for (int i = 0; i < n; ++i) res[i] = rq[i].res;
    core.summary(sum, wall);
    if (rc != VR_OK) return rc;
    return core.failed ? VR_ERR_STATE : VR_OK;
}

static int vr_serve_open_body(vr_ctx *c, const vr_serve_config *cfg, vr_server **out);
extern "C" int vr_serve_open(vr_ctx *c, const vr_serve_config *cfg, vr_server **out) {
    return abi_guard([&] { return vr_serve_open_body(c, cfg, out); });
}
static int vr_serve_open_body(vr_ctx *c, const vr_serve_config *cfg, vr_server **out) {
    if (!c || !cfg || !out) return arg_fail("null argument");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 64) return arg_fail("max_inflight must be 1..64");
    *out = nullptr;
    bool any_streamed = false;
    for (auto &kv : c->cubes) any_streamed |= kv.second->streamed;
    int rc = serve_prepare(c, any_streamed);
    if (rc) return rc;
    std::unique_ptr<vr_server> s(new (std::nothrow) vr_server());
    if (!s) return fail(VR_ERR_OOM, "no host memory for the server");
    s->c = c;
    if ((rc = s->core.open(c, cfg->max_inflight)) != VR_OK) {
        s->core.close();
        return rc;
    }
    try {
        s->th = std::thread([srv = s.get()]() { srv->run(); });
    } catch (...) {
        s->core.close();
        return fail(VR_ERR_OOM, "could not start the serving thread");
    }
    *out = s.release();
    return VR_OK;
}

static int vr_serve_submit_body(vr_server *s, const vr_request *req, int64_t *ticket);
extern "C" int vr_serve_submit(vr_server *s, const vr_request *req, int64_t *ticket) {
    return abi_guard([&] { return vr_serve_submit_body(s, req, ticket); });
}
static int vr_serve_submit_body(vr_server *s, const vr_request *req, int64_t *ticket) {
    if (!s || !req || !ticket) return arg_fail("null argument");
    try {
        std::unique_ptr<Req> r(new Req());
        const int rc = make_req(s->c, *req, *r);
        if (rc != VR_OK) return rc;
        Req *p = r.get();
        std::lock_guard<std::mutex> l(s->mu);
        if (s->closing) return fail(VR_ERR_STATE, "the server is closing");
        if (s->broken) return fail(VR_ERR_STATE, "the server's loop stopped: " + s->broken_what);
        p->arrival_ms = s->core.now();
        p->ticket = s->next_ticket++;
        *ticket = p->ticket;
        s->owned.emplace(p->ticket, std::move(r));
        s->submitted.push_back(p);
        ++s->outstanding;
        return VR_OK;
    } catch (const std::bad_alloc &) {
        return fail(VR_ERR_OOM, "no host memory for the request");
    }
}

static int vr_serve_poll_body(vr_server *s, int64_t *tickets, vr_request_result *results, int cap, int *n,
                             int wait_ms);
extern "C" int vr_serve_poll(vr_server *s, int64_t *tickets, vr_request_result *results, int cap, int *n,
                             int wait_ms) {
    return abi_guard([&] { return vr_serve_poll_body(s, tickets, results, cap, n, wait_ms); });
}
static int vr_serve_poll_body(vr_server *s, int64_t *tickets, vr_request_result *results, int cap, int *n,
                             int wait_ms) {
    if (!s || !n || (cap > 0 && (!tickets || !results))) return arg_fail("null argument");
    if (cap < 0 || wait_ms < 0 || wait_ms > 60000) return arg_fail("cap >= 0 and 0 <= wait_ms <= 60000");
    std::unique_lock<std::mutex> l(s->mu);
    if (s->completed.empty() && wait_ms > 0)
        s->cv.wait_for(l, std::chrono::milliseconds(wait_ms), [s]() { return !s->completed.empty(); });
    int k = 0;
    while (k < cap && !s->completed.empty()) {
        Req *r = s->completed.front();
        s->completed.pop_front();
        tickets[k] = r->ticket;
        results[k] = r->res;
        s->owned.erase(r->ticket);
        ++k;
    }
    *n = k;
    return VR_OK;
}

static int vr_serve_close_body(vr_server *s, vr_serve_summary *sum);
extern "C" int vr_serve_close(vr_server *s, vr_serve_summary *sum) {
    return abi_guard([&] { return vr_serve_close_body(s, sum); });
}
static int vr_serve_close_body(vr_server *s, vr_serve_summary *sum) {
    if (!s) return arg_fail("null argument");
    {
        std::lock_guard<std::mutex> l(s->mu);
        s->closing = true;
    }
    if (s->th.joinable()) s->th.join();
    const double wall = s->core.now();
    s->core.close();
    s->core.summary(sum, wall);
    const int rc = s->core.failed ? VR_ERR_STATE : VR_OK;
    delete s;
    return rc;
}
#pragma GCC visibility pop
