// vr_api.cu -- the C ABI of libvrcube.so (include/vrcube.h): context, cubes, bricking, and the
// per-frame host work-list (rendering rectangles, culling, front-to-back order, screen bins).
//
// Section 2.3 gives the call sequence (load, min/max, colour map, render requests with the
// view matrices); Section 2.4 the rendering rectangle of each part (here: the screen bounding
// box of each brick's projected corners); Section 2.5 the depth-ordered compositing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "vr_host.h"

using namespace vr;
using namespace vrh;

namespace vrh {

int set_dev(vr_ctx *c) {
    CK(cudaSetDevice(c->device));
    return VR_OK;
}

void layout_strides(const int dim[3], int layout, int str[3]) {
    // the contiguous axis first, then the other two in x, y, z order
    int ord[3];
    ord[0] = layout;
    for (int a = 0, k = 1; a < 3; ++a)
        if (a != layout) ord[k++] = a;
    int s = 1;
    for (int k = 0; k < 3; ++k) {
        str[ord[k]] = s;
        s *= dim[ord[k]];
    }
}

long long layout_strides_padded(const int dim[3], int a, int esz, int str[3]) {
    const int per16 = 16 / esz;
    const long long row = ((long long)dim[a] + per16 - 1) / per16 * per16;
    int ord[3];
    ord[0] = a;
    for (int q = 0, k = 1; q < 3; ++q)
        if (q != a) ord[k++] = q;
    str[ord[0]] = 1;
    str[ord[1]] = (int)row;
    str[ord[2]] = (int)(row * dim[ord[1]]);
    return row * dim[ord[1]] * dim[ord[2]];
}

FrameLayout frame_layout(const vr_ctx *c, const Cube *cb) {
    FrameLayout f{0, 0, kRcLong, kRcShort, 0.0f, 0};
    float best = -1.0f;
    // resident cubes: atlases built with the pool; streamed and compressed cubes: atlases of the
    // brick cache's slots, packed as bricks become resident
    const bool atlas = cb->streamed ? (cb->layouts & 8) != 0 : !cb->atlas_tex.empty();
    // with atlases, the image axis is fixed first: the one with the smaller z component
    const int only = atlas ? (std::fabs(c->cam.R[5]) < std::fabs(c->cam.R[2]) ? 1 : 0) : -1;
    for (int i = 0; i < 2; ++i)              // image axis: camera right (row 0), up (row 1)
        for (int a = 0; a < 3; ++a) {
            if (only >= 0 && i != only) continue;
            if (!(cb->layouts & (1 << a))) continue;
            const float sc = std::fabs(c->cam.R[3 * i + a]);
            if (sc > best + 1e-6f) {
                best = sc;
                f.layout = a;
                f.lanes_y = i;
            }
        }
    f.tw = f.lanes_y ? kRcShort : kRcLong;
    f.th = f.lanes_y ? kRcLong : kRcShort;
    f.align = best;
    f.atlas = atlas ? 1 : 0;
    return f;
}

void alpha_prefix(const vr_ctx *c, std::vector<int> &pre) {
    pre.assign(c->lut.size() + 1, 0);
    for (size_t i = 0; i < c->lut.size(); ++i) pre[i + 1] = pre[i] + (c->lut[i].w != 0.0f ? 1 : 0);
}

// A DVR sample's opacity interpolates table entries floor(x) and floor(x)+1 at
// x = clamp((v - vmin)/(vmax - vmin), 0, 1) (n - 1), and a trilinear value lies within its
// stencil's range, so a brick whose stored values map only to entries of zero opacity adds
// exactly nothing (every sample has a = 0: colour += T*0, T *= 1).  The range is widened for
// the FP32 rounding of the mapping and, for 16-bit bricks, for the rounding of the codes.
bool window_clip(const vr_ctx *c, const Cube *cb, const DrawBrick &b, float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = b.lo[a];
        hi[a] = b.hi[a];
        if (c->has_window) {
            lo[a] = std::max(lo[a], (float)std::max<int64_t>(c->win_lo[a], 0));
            hi[a] = std::min(hi[a], (float)std::min<int64_t>(c->win_hi[a], cb->n[a]));
        }
        if (!(hi[a] > lo[a])) return false;
    }
    return true;
}

bool skip_brick(const vr_ctx *c, const Cube *cb, size_t b, const int *pre) {
    if (c->mode != VR_DVR || c->full_rect || b >= cb->vlo.size()) return false;
    double lo = cb->vlo[b], hi = cb->vhi[b];
    if (!c->chmask.empty()) {                // disabled channels hold vmin
        lo = std::min(lo, (double)c->vmin);
        hi = std::max(hi, (double)c->vmin);
    }
    if (!(lo <= hi)) return false;
    const double mag = std::max({1.0, std::fabs(lo), std::fabs(hi)});
    const double widen = mag * (cb->storage == VR_F32 ? 1e-5 : 1.0 / 64.0);
    const double n1 = (double)c->lut.size() - 1.0;
    auto x_of = [&](double v) {
        const double u = (v - (double)c->vmin) / ((double)c->vmax - (double)c->vmin);
        return std::min(std::max(u, 0.0), 1.0) * n1;
    };
    const double xl = x_of(lo - widen) - 1e-3, xh = x_of(hi + widen) + 1e-3;
    const long i0 = std::max(0L, (long)std::floor(xl));
    const long i1 = std::min((long)n1, (long)std::floor(xh) + 1);
    return pre[i1 + 1] - pre[i0] == 0;
}

// Estimated ray-cast cost of brick bi for the current camera: the samples a full bundle of the
// frame's rays takes through it, its (window-clipped) core volume over the volume one sample
// stands for (a pixel's footprint at the brick's depth times the step); 0 when it is skipped
// (empty space), clipped away or projects entirely outside the frame.  Early termination is
// not modelled.
double brick_cost(const vr_ctx *c, const Cube *cb, size_t bi, const int *apre) {
    const DrawBrick &b = cb->tmpl[bi];
    float lo[3], hi[3];
    if (!window_clip(c, cb, b, lo, hi) || skip_brick(c, cb, bi, apre)) return 0.0;
    const Cam &m = c->cam;
    double vol = 1.0, ctr[3], diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        vol *= (double)hi[a] - lo[a];
        ctr[a] = 0.5 * ((double)lo[a] + hi[a]);
        diag2 += ((double)hi[a] - lo[a]) * ((double)hi[a] - lo[a]);
    }
    // projected extent (the corners' image-plane box) against the frame
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
    bool behind = false;
    for (int k = 0; k < 8; ++k) {
        const double q[3] = {(k & 1) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 4) ? hi[2] : lo[2]};
        double e[3];
        for (int r = 0; r < 3; ++r) e[r] = m.R[3 * r] * q[0] + m.R[3 * r + 1] * q[1] + m.R[3 * r + 2] * q[2] + m.t[r];
        double sx, sy;
        if (m.proj == VR_PERSP) {
            if (e[2] > -1e-6) { behind = true; continue; }
            sx = e[0] / (-e[2]) / m.th_w;
            sy = e[1] / (-e[2]) / m.th;
        } else {
            sx = e[0] / m.half_w;
            sy = e[1] / m.half_h;
        }
        mnx = std::min(mnx, sx); mxx = std::max(mxx, sx);
        mny = std::min(mny, sy); mxy = std::max(mxy, sy);
    }
    if (!behind && (mxx < -1.0 || mnx > 1.0 || mxy < -1.0 || mny > 1.0)) return 0.0;
    double pix;
    if (m.proj == VR_PERSP) {
        const double ez = m.R[6] * ctr[0] + m.R[7] * ctr[1] + m.R[8] * ctr[2] + m.t[2];
        const double depth = std::max(-ez, 0.5 * std::sqrt(diag2));
        pix = 2.0 * depth * m.th / m.H;
    } else {
        pix = 2.0 * m.half_h / m.H;
    }
    return vol / (pix * pix * (double)c->step);
}

// Recursive longest-axis split (Section 2.2, Fig. 3): at every level the current part's brick
// range is cut along its longest axis (in voxels; ties to the lower axis) into counts[L]
// consecutive slabs of whole brick layers and the path keeps slab index[L].  Equal split: as
// even a layer count as possible.  Balanced split (Section 3: the slowest GPU sets the frame
// time, and the work of a part depends on the view): the cuts fall where the cumulative
// estimated cost of the part's layers for the current camera crosses k/counts[L] of its total,
// each slab keeping at least one layer while layers last.  A part may be empty when a level has
// more slabs than layers.
PartBox partition_box(const vr_ctx *c, const Cube *cb) {
    PartBox p{};
    for (int a = 0; a < 3; ++a) { p.lo[a] = 0; p.hi[a] = (int)cb->nb[a]; }
    const bool balanced = cb->part_balance && c->cam_set && c->tf_set && cb->part_nlev > 0;
    // the bricks' costs depend on the camera, table, parameters, window and bricking, not on the
    // part: computed once per render state and reused by every rank's part and compositing stage
    const uint64_t key = c->state_gen - c->part_gen;
    if (balanced && (cb->cost_key != key || cb->cost_cache.size() != cb->tmpl.size())) {
        std::vector<int> apre;
        alpha_prefix(c, apre);
        cb->cost_cache.resize(cb->tmpl.size());
        for (size_t bi = 0; bi < cb->tmpl.size(); ++bi) cb->cost_cache[bi] = brick_cost(c, cb, bi, apre.data());
        cb->cost_key = key;
    }
    const std::vector<double> &cost = cb->cost_cache;
    for (int L = 0; L < cb->part_nlev; ++L) {
        int axis = 0;
        int64_t best = -1;
        for (int a = 0; a < 3; ++a) {
            const int64_t ext = std::min<int64_t>((int64_t)p.hi[a] * cb->B[a], cb->n[a]) - (int64_t)p.lo[a] * cb->B[a];
            if (ext > best) { best = ext; axis = a; }
        }
        const int64_t layers = p.hi[axis] - p.lo[axis], n = cb->part_counts[L], k = cb->part_index[L];
        int s0 = p.lo[axis] + (int)(layers * k / n), s1 = p.lo[axis] + (int)(layers * (k + 1) / n);
        if (balanced && layers > 0) {
            // cost of each layer of the current part along the axis
            std::vector<double> lc((size_t)layers, 0.0);
            for (size_t bi = 0; bi < cb->tmpl.size(); ++bi) {
                const int64_t ci[3] = {(int64_t)bi % cb->nb[0], ((int64_t)bi / cb->nb[0]) % cb->nb[1],
                                       (int64_t)bi / (cb->nb[0] * cb->nb[1])};
                bool in = true;
                for (int a = 0; a < 3; ++a) in = in && ci[a] >= p.lo[a] && ci[a] < p.hi[a];
                if (in) lc[(size_t)(ci[axis] - p.lo[axis])] += cost[bi];
            }
            double total = 0.0;
            for (double v : lc) total += v;
            // cut j (1..n-1): the first layer boundary where the prefix cost reaches j/n of the
            // total, kept strictly increasing while layers last
            std::vector<int64_t> cut((size_t)n + 1, 0);
            cut[(size_t)n] = layers;
            double pre = 0.0;
            int64_t li = 0;
            for (int64_t j = 1; j < n; ++j) {
                const double target = total * (double)j / (double)n;
                while (li < layers && pre + lc[(size_t)li] * 0.5 < target) pre += lc[(size_t)li++];
                const int64_t lo_ok = std::min<int64_t>(cut[(size_t)j - 1] + 1, layers);
                cut[(size_t)j] = std::min<int64_t>(std::max<int64_t>(li, lo_ok), layers);
            }
            for (int64_t j = n - 1; j >= 1; --j)        // leave room for the later slabs
                cut[(size_t)j] = std::min<int64_t>(cut[(size_t)j], std::max<int64_t>(layers - (n - j), 0));
            s0 = p.lo[axis] + (int)cut[(size_t)k];
            s1 = p.lo[axis] + (int)cut[(size_t)k + 1];
            if (s1 < s0) s1 = s0;
        }
        p.axis[L] = axis;
        p.lo[axis] = s0;
        p.hi[axis] = s1;
    }
    return p;
}

bool in_part(const PartBox &p, const Cube *cb, int64_t brick) {
    const int64_t ci[3] = {brick % cb->nb[0], (brick / cb->nb[0]) % cb->nb[1], brick / (cb->nb[0] * cb->nb[1])};
    for (int a = 0; a < 3; ++a)
        if (ci[a] < p.lo[a] || ci[a] >= p.hi[a]) return false;
    return true;
}

Cube *find_cube(vr_ctx *c, int id) {
    auto it = c->cubes.find(id);
    return it == c->cubes.end() ? nullptr : it->second;
}

int ensure_host(vr_ctx *c, size_t bytes) {
    if (c->h_cap >= bytes && c->h_stage) return VR_OK;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    if (c->h_stage) CK(cudaFreeHost(c->h_stage));
    c->h_stage = nullptr;
    size_t want = std::max(bytes, c->h_cap * 3 / 2);
    CK(cudaMallocHost(&c->h_stage, want));
    c->h_cap = want;
    return VR_OK;
}

// ---------------------------------------------------------------------------------------------
// per-frame work-list
// ---------------------------------------------------------------------------------------------

// World position of the perspective eye in the renderer's FP32 arithmetic (R^T (0 - t)); every
// perspective ray starts exactly there.
void eye_f32(const Cam &c, float o[3]) {
    volatile float y0 = 0.0f - c.t[0], y1 = 0.0f - c.t[1], y2 = 0.0f - c.t[2];
    for (int k = 0; k < 3; ++k) {
        volatile float a = c.R[k] * y0;
        volatile float b = c.R[3 + k] * y1;
        volatile float s = a + b;
        volatile float d = c.R[6 + k] * y2;
        volatile float r = s + d;
        o[k] = r;
    }
}

void build_worklist(vr_ctx *c, Cube *cb, WorkList &wl) {
    const Cam &cam = c->cam;
    const int W = cam.W, H = cam.H;
    const double R[9] = {cam.R[0], cam.R[1], cam.R[2], cam.R[3], cam.R[4], cam.R[5], cam.R[6], cam.R[7], cam.R[8]};
    const double t[3] = {cam.t[0], cam.t[1], cam.t[2]};
    // ordering reference: the perspective eye's cell, or the orthographic direction
    int ecell[3] = {0, 0, 0};
    int dsign[3] = {1, 1, 1};
    if (cam.proj == VR_PERSP) {
        float e[3];
        eye_f32(cam, e);
        for (int a = 0; a < 3; ++a) {
            if (e[a] < 0.0f) ecell[a] = -1;
            else if (e[a] >= (float)cb->n[a]) ecell[a] = (int)cb->nb[a];
            else ecell[a] = std::min((int)(e[a] / (float)cb->B[a]), (int)cb->nb[a] - 1);
            // e >= lo of that cell holds: a cell index is floor(e / B) for exact integers lo
            while (ecell[a] > 0 && ecell[a] < cb->nb[a] && (float)((int64_t)ecell[a] * cb->B[a]) > e[a]) --ecell[a];
            while (ecell[a] + 1 < cb->nb[a] && (float)((int64_t)(ecell[a] + 1) * cb->B[a]) <= e[a]) ++ecell[a];
        }
    } else {
        for (int a = 0; a < 3; ++a) dsign[a] = (-cam.R[6 + a] >= 0.0f) ? 1 : -1;   // d = -R row 2
    }
    std::vector<std::pair<long long, int>> order;
    std::vector<DrawBrick> cand;
    cand.reserve(cb->tmpl.size());
    std::vector<int> apre;
    alpha_prefix(c, apre);
    const bool parted = cb->part_nlev > 0;      // bricks outside the cube's part are not drawn
    const PartBox part = parted ? partition_box(c, cb) : PartBox{};
    for (size_t bi = 0; bi < cb->tmpl.size(); ++bi) {
        DrawBrick b = cb->tmpl[bi];
        if (parted && !in_part(part, cb, (int64_t)bi)) continue;
        if (!window_clip(c, cb, b, b.lo, b.hi)) continue;
        if (skip_brick(c, cb, bi, apre.data())) continue;
        int x0 = 0, y0 = 0, x1 = W, y1 = H;
        bool cull = false;
        if (!c->full_rect) {
            double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
            int behind = 0, front = 0;
            for (int k = 0; k < 8; ++k) {
                double p[3] = {(k & 1) ? b.hi[0] : b.lo[0], (k & 2) ? b.hi[1] : b.lo[1], (k & 4) ? b.hi[2] : b.lo[2]};
                double e[3];
                for (int r = 0; r < 3; ++r) e[r] = R[3 * r] * p[0] + R[3 * r + 1] * p[1] + R[3 * r + 2] * p[2] + t[r];
                double sx, sy;
                if (cam.proj == VR_PERSP) {
                    if (e[2] > -1e-6) { ++behind; continue; }
                    ++front;
                    sx = e[0] / (-e[2]) / cam.th_w;
                    sy = e[1] / (-e[2]) / cam.th;
                } else {
                    if (e[2] > 0.0) ++behind; else ++front;
                    sx = e[0] / cam.half_w;
                    sy = e[1] / cam.half_h;
                }
                double px = (sx + 1.0) * 0.5 * W, py = (1.0 - sy) * 0.5 * H;
                mnx = std::min(mnx, px); mxx = std::max(mxx, px);
                mny = std::min(mny, py); mxy = std::max(mxy, py);
            }
            if (front == 0) {
                cull = true;                       // entirely behind the eye / image plane
            } else if (cam.proj == VR_PERSP && behind > 0) {
                x0 = 0; y0 = 0; x1 = W; y1 = H;     // straddles the eye plane: whole frame
            } else {
                // clamped to the frame in double first: the int conversion of an
                // out-of-range double is undefined
                x0 = (int)std::min((double)W, std::max(0.0, std::floor(mnx) - 1.0));
                y0 = (int)std::min((double)H, std::max(0.0, std::floor(mny) - 1.0));
                x1 = (int)std::max(0.0, std::min((double)W, std::ceil(mxx) + 1.0));
                y1 = (int)std::max(0.0, std::min((double)H, std::ceil(mxy) + 1.0));
                if (x1 <= x0 || y1 <= y0) cull = true;
            }
        }
        if (cull) continue;
        DrawBrick d = b;
        d.rect[0] = x0; d.rect[1] = y0; d.rect[2] = x1 - x0; d.rect[3] = y1 - y0;
        d.sampled = 0;
        int cidx[3] = {(int)(b.brick % cb->nb[0]), (int)((b.brick / cb->nb[0]) % cb->nb[1]),
                       (int)(b.brick / (cb->nb[0] * cb->nb[1]))};
        long long key = 0;
        for (int a = 0; a < 3; ++a) {
            if (cam.proj == VR_PERSP) key += std::abs(cidx[a] - ecell[a]);
            else key += dsign[a] > 0 ? cidx[a] : (cb->nb[a] - 1 - cidx[a]);
        }
        order.push_back({key, (int)cand.size()});
        cand.push_back(d);
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) { return a.first < b.first; });
    wl.db.clear();
    wl.items.clear();
    wl.db.reserve(order.size());
    const FrameLayout fl = frame_layout(c, cb);
    long long frag = 0;
    for (auto &o : order) {
        DrawBrick d = cand[o.second];
        d.frag_off = frag;
        frag += (long long)d.rect[2] * d.rect[3];
        if (!cb->loff.empty()) d.data_off = cb->loff[3 * (size_t)d.brick + fl.layout];
        layout_strides(d.dim, fl.layout, d.str);
        d.pad_off = -1;
        if (!cb->loff_pad.empty() && cb->loff_pad[3 * (size_t)d.brick + fl.layout] >= 0) {
            d.pad_off = cb->loff_pad[3 * (size_t)d.brick + fl.layout];
            layout_strides_padded(d.dim, fl.layout, cb->storage == VR_F32 ? 4 : 2, d.pad_str);
        }
        int tw = (d.rect[2] + fl.tw - 1) / fl.tw, th = (d.rect[3] + fl.th - 1) / fl.th;
        int di = (int)wl.db.size();
        for (int ty = 0; ty < th; ++ty)
            for (int tx = 0; tx < tw; ++tx) wl.items.push_back(TileItem{di, tx, ty});
        wl.db.push_back(d);
    }
    wl.frag_px = frag;
    // screen-tile bins in front-to-back order
    const int ntx = (W + kTile - 1) / kTile, nty = (H + kTile - 1) / kTile;
    wl.tile_start.assign((size_t)ntx * nty + 1, 0);
    for (auto &d : wl.db) {
        int tx0 = d.rect[0] / kTile, tx1 = (d.rect[0] + d.rect[2] - 1) / kTile;
        int ty0 = d.rect[1] / kTile, ty1 = (d.rect[1] + d.rect[3] - 1) / kTile;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) wl.tile_start[(size_t)ty * ntx + tx + 1]++;
    }
    for (size_t i = 1; i < wl.tile_start.size(); ++i) wl.tile_start[i] += wl.tile_start[i - 1];
    wl.tile_list.assign(wl.tile_start.back(), 0);
    std::vector<int> fill(wl.tile_start.begin(), wl.tile_start.end() - 1);
    for (size_t di = 0; di < wl.db.size(); ++di) {
        const DrawBrick &d = wl.db[di];
        int tx0 = d.rect[0] / kTile, tx1 = (d.rect[0] + d.rect[2] - 1) / kTile;
        int ty0 = d.rect[1] / kTile, ty1 = (d.rect[1] + d.rect[3] - 1) / kTile;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) wl.tile_list[fill[(size_t)ty * ntx + tx]++] = (int)di;
    }
    // layout of the staged upload
    size_t off = 0;
    wl.off_lut = off; off = align_up(off + sizeof(float4) * c->lut.size(), 256);
    wl.off_db = off; off = align_up(off + sizeof(DrawBrick) * wl.db.size(), 256);
    wl.off_items = off; off = align_up(off + sizeof(TileItem) * wl.items.size(), 256);
    wl.off_ts = off; off = align_up(off + sizeof(int) * wl.tile_start.size(), 256);
    wl.off_tl = off; off = align_up(off + sizeof(int) * wl.tile_list.size(), 256);
    wl.off_mask = off; off = align_up(off + c->chmask.size(), 256);
    wl.bytes = off;
}

FrameConsts make_consts(vr_ctx *c, Cube *cb) {
    FrameConsts fc{};
    fc.cam = c->cam;
    fc.step = c->step;
    volatile float one_minus = 1.0f - std::min(c->tau, 1.0f);
    fc.thr = one_minus;
    fc.vmin = c->vmin;
    fc.inv_range = (float)(1.0 / ((double)c->vmax - (double)c->vmin));
    fc.lutmax = (float)(c->lut.size() - 1);
    fc.nlut = (int)c->lut.size();
    fc.mode = c->mode;
    fc.storage = cb->storage;
    fc.nx = (int)cb->n[0]; fc.ny = (int)cb->n[1]; fc.nz = (int)cb->n[2];
    const FrameLayout fl = frame_layout(c, cb);
    fc.lanes_y = fl.lanes_y;
    // atlases: two gathers per sample.  Linear copies: with a warp's rays along the contiguous
    // axis its loads are nearly coalesced and the stencil cache's bookkeeping costs more than
    // it saves; with a poor alignment it pays
    fc.fetch = fl.atlas ? (cb->atlas_pair && !cb->streamed ? 5 : 2) : (fl.align < 0.9f ? 1 : 0);
    fc.sub = c->subimage ? 1 : 0;
    // staged slabs: DVR frames of resident FP32 cubes that keep the padded copy of the frame
    // layout; the march axis is the view's dominant axis other than the contiguous one
    if ((cb->layouts & 16) && !cb->streamed && c->mode == VR_DVR && cb->storage == VR_F32 &&
        !cb->loff_pad.empty() && cb->loff_pad[fl.layout] >= 0) {
        const float fwd[3] = {-c->cam.R[6], -c->cam.R[7], -c->cam.R[8]};
        int m = -1;
        for (int a = 0; a < 3; ++a)
            if (a != fl.layout && (m < 0 || std::fabs(fwd[a]) > std::fabs(fwd[m]))) m = a;
        if (std::fabs(fwd[m]) > 0.3f) {
            fc.fetch = 4;
            fc.stage_m = m;
            fc.stage_dir = fwd[m] > 0.0f ? 1 : -1;
        }
    }
    return fc;
}

// Camera constants of a view (validated): rotation rows and translation from the row-major
// world -> eye matrix, half extents (orthographic) or tan(fov / 2) (perspective), each rounded
// to binary32 once.
int make_cam(const float view[16], int proj, float param, int width, int height, Cam &cam) {
    if (proj != VR_ORTHO && proj != VR_PERSP) return arg_fail("bad projection");
    if (width < 1 || height < 1 || width > 16384 || height > 16384) return arg_fail("bad frame size");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(view[i])) return arg_fail("non-finite view matrix");
    if (!(param > 0.0f) || !std::isfinite(param)) return arg_fail("bad projection parameter");
    if (proj == VR_PERSP && !(param < 3.14159f)) return arg_fail("fov must be < pi");
    // the rotation part must be (close to) orthonormal: rays need a unit direction
    double det = (double)view[0] * ((double)view[5] * view[10] - (double)view[6] * view[9]) -
                 (double)view[1] * ((double)view[4] * view[10] - (double)view[6] * view[8]) +
                 (double)view[2] * ((double)view[4] * view[9] - (double)view[5] * view[8]);
    if (!(det > 0.5 && det < 2.0)) return arg_fail("view rotation is not a rotation");
    std::memset(&cam, 0, sizeof(cam));
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) cam.R[3 * r + k] = view[4 * r + k];
        cam.t[r] = view[4 * r + 3];
    }
    cam.proj = proj;
    cam.W = width;
    cam.H = height;
    volatile float aspect = (float)width / (float)height;
    volatile float hh = param * 0.5f;
    volatile float hw = hh * aspect;
    cam.half_h = hh;
    cam.half_w = hw;
    volatile float th = (float)std::tan((double)param * 0.5);
    volatile float thw = th * aspect;
    cam.th = th;
    cam.th_w = thw;
    return VR_OK;
}

// Preconditions of the gradient calls: DVR, resident FP32 bricks, per-segment termination.
int backward_ready(vr_ctx *c, Cube *cb) {
    int rc = check_ready(c, cb);
    if (rc) return rc;
    if (c->mode != VR_DVR || cb->storage != VR_F32 || cb->streamed)
        return fail(VR_ERR_UNSUPPORTED, "backward needs DVR mode and resident FP32 bricks");
    if (c->term != VR_TERM_SEGMENT)
        return fail(VR_ERR_UNSUPPORTED, "backward replays per-segment termination (VR_TERM_SEGMENT)");
    return VR_OK;
}

// The adjoint of the current camera's frame: composite backward, ray replay, and the table
// gradient either reduced into grad_lut (FP64 sum rounded once) or, with acc, added to the FP64
// accumulator of a batch of views (zeroed first when `first`).
int backward_view(vr_ctx *c, Cube *cb, const float *grad_out, float *grad_lut, double *acc, bool first,
                  float *grad_voxels, cudaStream_t s) {
    int rc;
    FrameConsts fc = make_consts(c, cb);
    WorkList wl;
    if ((rc = stage_frame(c, cb, wl, s, nullptr)) != VR_OK) return rc;
    if (!c->chmask.empty()) fc.chmask = reinterpret_cast<const unsigned char *>(c->d_stage.p + wl.off_mask);
    const size_t nfr = (size_t)std::max<long long>(wl.frag_px, 1);
    const char *frags_before = c->d_frags.p;
    if ((rc = ensure(c->d_frags, nfr * sizeof(float4), c)) != VR_OK) return rc;
    if ((rc = ensure(c->d_gfrag, nfr, c)) != VR_OK) return rc;
    // the last frame's fragments are this frame's when nothing that changes a frame was called
    // since and no other frame wrote them (the common render-then-backward step)
    const bool reuse = c->frag_valid && c->frag_cube == cb->id && c->frag_gen == c->state_gen &&
                       c->d_frags.p == frags_before;
    const int nitems = (int)wl.items.size();
    if ((rc = ensure(c->d_gpart, (size_t)std::max(nitems, 1) * 4 * fc.nlut, c)) != VR_OK) return rc;
    if ((rc = ensure(c->d_gchunk, (size_t)kLutGradChunks * 4 * fc.nlut, c)) != VR_OK) return rc;
    char *d = c->d_stage.p;
    const float4 *d_lut = reinterpret_cast<const float4 *>(d + wl.off_lut);
    const DrawBrick *d_db = reinterpret_cast<const DrawBrick *>(d + wl.off_db);
    const TileItem *d_items = reinterpret_cast<const TileItem *>(d + wl.off_items);
    const int *d_ts = reinterpret_cast<const int *>(d + wl.off_ts);
    const int *d_tl = reinterpret_cast<const int *>(d + wl.off_tl);
    if (!reuse) {
        c->frag_valid = false;
        CK(launch_raycast(fc, d_lut, d_db, d_items, nitems, cb->d_pool, c->d_frags.p, c->d_ctr, s));
        c->frag_valid = true;
        c->frag_cube = cb->id;
        c->frag_gen = c->state_gen;
    }
    CK(launch_composite_backward(fc, d_db, d_ts, d_tl, reinterpret_cast<const float4 *>(c->d_frags.p),
                                 reinterpret_cast<const float4 *>(grad_out), c->d_gfrag.p, s));
    if (nitems > 0)
        CK(launch_adjoint(fc, d_lut, d_db, d_items, nitems, static_cast<const float *>(cb->d_pool),
                          reinterpret_cast<const float4 *>(c->d_frags.p), c->d_gfrag.p, c->d_gpart.p,
                          grad_voxels, s));
    if (acc) {
        CK(launch_lut_grad_accumulate(c->d_gpart.p, nitems, fc.nlut, c->d_gchunk.p, acc, first, s));
    } else if (nitems > 0) {
        CK(launch_lut_grad_reduce(c->d_gpart.p, nitems, fc.nlut, c->d_gchunk.p, grad_lut, s));
    } else {
        CK(cudaMemsetAsync(grad_lut, 0, sizeof(float) * 4 * fc.nlut, s));
    }
    CK(cudaEventRecord(c->frame_done, s));
    c->frame_pending = true;
    return VR_OK;
}

int timing_events(vr_ctx *c, cudaEvent_t ev[4]) {
    for (int i = 0; i < 4; ++i) {
        if (c->ev_pool.empty()) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->ev_pool.push_back(e);
        }
        ev[i] = c->ev_pool.back();
        c->ev_pool.pop_back();
    }
    return VR_OK;
}

int collect_timing(vr_ctx *c) {
    for (auto &ev : c->ev_pending) {
        CK(cudaEventSynchronize(ev[3]));
        float a = 0, b = 0, f = 0;
        CK(cudaEventElapsedTime(&a, ev[1], ev[2]));
        CK(cudaEventElapsedTime(&b, ev[2], ev[3]));
        CK(cudaEventElapsedTime(&f, ev[0], ev[3]));
        c->ms_raycast += a;
        c->ms_composite += b;
        c->ms_frame += f;
        c->timed_frames++;
        for (auto e : ev) c->ev_pool.push_back(e);
    }
    c->ev_pending.clear();
    return VR_OK;
}

// Stages the work-list (table, bricks, items, bins) and uploads it on `s`.
int stage_frame(vr_ctx *c, Cube *cb, WorkList &wl, cudaStream_t s, cudaEvent_t ev0) {
    build_worklist(c, cb, wl);
    // the previous frame must be done with the pinned staging and the device scratch
    if (c->frame_pending) {
        CK(cudaEventSynchronize(c->upload_done));
        CK(cudaStreamWaitEvent(s, c->frame_done, 0));
    }
    int rc;
    if ((rc = ensure_host(c, wl.bytes)) != VR_OK) return rc;
    if ((rc = ensure(c->d_stage, wl.bytes, c)) != VR_OK) return rc;
    char *h = c->h_stage;
    std::memcpy(h + wl.off_lut, c->lut.data(), sizeof(float4) * c->lut.size());
    if (!wl.db.empty()) std::memcpy(h + wl.off_db, wl.db.data(), sizeof(DrawBrick) * wl.db.size());
    if (!wl.items.empty()) std::memcpy(h + wl.off_items, wl.items.data(), sizeof(TileItem) * wl.items.size());
    std::memcpy(h + wl.off_ts, wl.tile_start.data(), sizeof(int) * wl.tile_start.size());
    if (!wl.tile_list.empty()) std::memcpy(h + wl.off_tl, wl.tile_list.data(), sizeof(int) * wl.tile_list.size());
    if (!c->chmask.empty()) std::memcpy(h + wl.off_mask, c->chmask.data(), c->chmask.size());
    if (ev0) CK(cudaEventRecord(ev0, s));
    CK(cudaMemcpyAsync(c->d_stage.p, h, wl.bytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->upload_done, s));
    return VR_OK;
}

int check_ready(vr_ctx *c, Cube *cb) {
    if (!cb->bricked) { g_last_error = "cube has no bricking"; return VR_ERR_STATE; }
    if (!c->chmask.empty() && (int64_t)c->chmask.size() != cb->n[2])
        return arg_fail("the channel mask must have one entry per z of the cube");
    if (!c->tf_set) { g_last_error = "no transfer function"; return VR_ERR_STATE; }
    if (!c->cam_set) { g_last_error = "no camera"; return VR_ERR_STATE; }
    // every lattice index k = t/step reached inside the cube must fit comfortably in an int:
    // t <= |camera - cube centre| + half diagonal
    const Cam &m = c->cam;
    double eye[3], cen[3], dist2 = 0.0, diag2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        eye[k] = -((double)m.R[k] * m.t[0] + (double)m.R[3 + k] * m.t[1] + (double)m.R[6 + k] * m.t[2]);
        cen[k] = 0.5 * (double)cb->n[k];
        dist2 += (eye[k] - cen[k]) * (eye[k] - cen[k]);
        diag2 += (double)cb->n[k] * cb->n[k];
    }
    const double tmax = std::sqrt(dist2) + std::sqrt(diag2);
    if (tmax / (double)c->step > (double)(1 << 28) || std::sqrt(diag2) / c->step > (double)(1 << 24))
        return arg_fail("step too small for this camera and cube (lattice index would overflow)");
    return VR_OK;
}

// Releases a cube's slice atlases.  Frames in flight may still gather from them: the device is
// drained first (atlases change only with the bricking or the voxels).
void free_atlases(Cube *cb) {
    if (cb->atlas_arr.empty() && cb->atlas_tex.empty()) return;
    cudaDeviceSynchronize();
    for (auto t : cb->atlas_tex)
        if (t) cudaDestroyTextureObject(t);
    for (auto a : cb->atlas_arr)
        if (a) cudaFreeArray(a);
    cb->atlas_tex.clear();
    cb->atlas_arr.clear();
    cb->atlas_bytes = 0;
    cb->atlas_pair = false;
    for (auto &d : cb->tmpl) { d.atlas = 0; d.alog = 0; }
}

// Slice atlas of every brick (layout bit 3) from its x-contiguous copy in the pool: slice z
// of a brick of dx x dy x dz stored elements becomes tile (z mod 2^alog, z div 2^alog) of a 2D
// array of 2^alog dx x ceil(dz / 2^alog) dy texels, with 2^alog the smallest power of two whose
// square is >= dz.  FP32 bricks keep their values, 16-bit bricks their codes (FP16 as half
// texels, BF16 as 16-bit unsigned ones).  With layout bit 5, 16-bit bricks get pair atlases
// instead: dz - 1 tiles of 32-bit texels, tile z holding the codes of slices z and z + 1 (one
// gather per sample).  The array must fit the device's limit for 2D gathers.
int build_atlases(vr_ctx *c, Cube *cb, cudaStream_t s) {
    free_atlases(cb);
    const int nbr = (int)cb->tmpl.size();
    const bool pair = (cb->layouts & 32) && cb->storage != VR_F32;
    const size_t bsz = cb->storage == VR_F32 ? 4 : 2;       // bytes of a stored element
    const size_t esz = pair ? 4 : bsz;                       // bytes of a texel
    int gw = 0, gh = 0;
    CK(cudaDeviceGetAttribute(&gw, cudaDevAttrMaxTexture2DGatherWidth, c->device));
    CK(cudaDeviceGetAttribute(&gh, cudaDevAttrMaxTexture2DGatherHeight, c->device));
    std::vector<int> lg(nbr);
    size_t most = 16;
    for (int i = 0; i < nbr; ++i) {
        const int *dm = cb->tmpl[i].dim;
        const int nt = pair ? dm[2] - 1 : dm[2];            // tiles
        int l = 0;
        while ((1ll << (2 * l)) < nt) ++l;
        const long long w = (long long)dm[0] << l, h = (long long)((nt + (1 << l) - 1) >> l) * dm[1];
        if (w > gw || h > gh) return fail(VR_ERR_UNSUPPORTED, "bricks too large for a slice atlas (2D gather limit)");
        lg[i] = l;
        most = std::max(most, (size_t)(w * h) * esz);
    }
    void *tmp = nullptr;
    CK(cudaMalloc(&tmp, most));
    std::vector<cudaSurfaceObject_t> surfs;   // kept until the packs that write through them ran
    auto bail = [&](cudaError_t e, const char *what) {
        cudaStreamSynchronize(s);
        for (auto sf : surfs) cudaDestroySurfaceObject(sf);
        cudaFree(tmp);
        free_atlases(cb);
        return cuda_fail(e, what);
    };
    cudaError_t e = cudaMemsetAsync(tmp, 0, most, s);
    if (e != cudaSuccess) return bail(e, "cudaMemsetAsync");
    // FP32 values; FP16 codes as half texels (gathers widen them to float exactly); BF16 codes as
    // 16-bit unsigned texels (widened in the kernel)
    // (pair atlases: two codes in one 32-bit unsigned texel, widened in the kernel)
    const cudaChannelFormatDesc cd = pair ? cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindUnsigned)
                                   : esz == 4 ? cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat)
                                   : cb->storage == VR_F16 ? cudaCreateChannelDescHalf()
                                                           : cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned);
    cb->atlas_arr.assign(nbr, nullptr);
    cb->atlas_tex.assign(nbr, 0);
    for (int i = 0; i < nbr; ++i) {
        const int *dm = cb->tmpl[i].dim;
        const int nt = pair ? dm[2] - 1 : dm[2];
        const size_t w = (size_t)dm[0] << lg[i], h = (size_t)((nt + (1 << lg[i]) - 1) >> lg[i]) * dm[1];
        cudaArray_t arr = nullptr;
        // written by the pack kernel through a surface where the device allows surface stores on
        // a gather array; else packed into staging and copied (the copy engine's array writes)
        const bool surf_ok = cudaMallocArray(&arr, &cd, w, h, cudaArrayTextureGather | cudaArraySurfaceLoadStore) ==
                             cudaSuccess;
        if (!surf_ok) {
            arr = nullptr;
            cudaGetLastError();
            if ((e = cudaMallocArray(&arr, &cd, w, h, cudaArrayTextureGather)) != cudaSuccess)
                return bail(e, "cudaMallocArray (slice atlas)");
        }
        cb->atlas_arr[i] = arr;
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        const char *src = static_cast<const char *>(cb->d_pool) + (size_t)cb->loff[3 * (size_t)i] * bsz;
        if (surf_ok) {
            cudaSurfaceObject_t sf = 0;
            if ((e = cudaCreateSurfaceObject(&sf, &rd)) != cudaSuccess) return bail(e, "cudaCreateSurfaceObject");
            surfs.push_back(sf);
            e = pair ? launch_pair_pack(src, dm[0], dm[1], dm[2], lg[i], nullptr, 0, (unsigned long long)sf, s)
                     : launch_atlas_pack_surf(src, (int)esz, dm[0], dm[1], dm[2], lg[i], (unsigned long long)sf, s);
            if (e != cudaSuccess) return bail(e, "atlas pack launch");
        } else {
            e = pair ? launch_pair_pack(src, dm[0], dm[1], dm[2], lg[i], tmp, w * esz, 0ull, s)
                     : launch_atlas_pack(src, (int)esz, dm[0], dm[1], dm[2], lg[i], tmp, w * esz, s);
            if (e != cudaSuccess) return bail(e, "atlas pack launch");
            if ((e = cudaMemcpy2DToArrayAsync(arr, 0, 0, tmp, w * esz, w * esz, h, cudaMemcpyDeviceToDevice, s)) !=
                cudaSuccess)
                return bail(e, "cudaMemcpy2DToArrayAsync (slice atlas)");
        }
        cudaTextureDesc td{};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        cudaTextureObject_t t = 0;
        if ((e = cudaCreateTextureObject(&t, &rd, &td, nullptr)) != cudaSuccess)
            return bail(e, "cudaCreateTextureObject (slice atlas)");
        cb->atlas_tex[i] = t;
        cb->atlas_bytes += w * h * esz;
        cb->tmpl[i].atlas = t;
        cb->tmpl[i].alog = lg[i];
    }
    e = cudaStreamSynchronize(s);
    for (auto sf : surfs) cudaDestroySurfaceObject(sf);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        free_atlases(cb);
        return cuda_fail(e, "slice atlas build");
    }
    cb->atlas_pair = pair;
    return VR_OK;
}

int build_bricks(vr_ctx *c, Cube *cb, cudaStream_t s) {
    const int nbr = (int)cb->tmpl.size();
    unsigned int *d_range = cb->d_bs + 2 * (size_t)nbr;
    // max |v| (16-bit scales) and the value range (empty-space skipping) of every brick
    CK(cudaMemsetAsync(cb->d_bs, 0, sizeof(unsigned int) * nbr, s));
    {
        std::vector<unsigned int> init(2 * (size_t)nbr);
        for (int i = 0; i < nbr; ++i) { init[2 * i] = 0xffffffffu; init[2 * i + 1] = 0u; }
        CK(cudaMemcpyAsync(d_range, init.data(), sizeof(unsigned int) * 2 * nbr, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(cb->d_tmpl, cb->tmpl.data(), sizeof(DrawBrick) * nbr, cudaMemcpyHostToDevice, s));
        CK(launch_brick_maxabs(cb->d_src, (int)cb->n[0], (int)cb->n[1], (int)cb->n[2], cb->d_tmpl, nbr, cb->d_bs,
                               d_range, s));
        std::vector<unsigned int> r(2 * (size_t)nbr);
        CK(cudaMemcpyAsync(r.data(), d_range, sizeof(unsigned int) * 2 * nbr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        auto dec = [](unsigned int e) {
            unsigned int b = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
            float f;
            std::memcpy(&f, &b, 4);
            return f;
        };
        cb->vlo.resize(nbr);
        cb->vhi.resize(nbr);
        for (int i = 0; i < nbr; ++i) { cb->vlo[i] = dec(r[2 * i]); cb->vhi[i] = dec(r[2 * i + 1]); }
    }
    int *d_exps = reinterpret_cast<int *>(cb->d_bs + nbr);
    // one build per kept layout: the records carry that layout's offsets and strides
    std::vector<DrawBrick> rec(cb->tmpl);
    for (int a = 0; a < 3; ++a) {
        if (!(cb->layouts & (1 << a))) continue;
        for (int i = 0; i < nbr; ++i) {
            rec[i].data_off = cb->loff[3 * (size_t)i + a];
            layout_strides(rec[i].dim, a, rec[i].str);
        }
        CK(cudaMemcpyAsync(cb->d_tmpl, rec.data(), sizeof(DrawBrick) * nbr, cudaMemcpyHostToDevice, s));
        CK(launch_brick_build(cb->d_src, (int)cb->n[0], (int)cb->n[1], (int)cb->n[2], cb->d_tmpl, nbr, cb->d_bs,
                              cb->storage, cb->d_pool, d_exps, s));
        CK(cudaStreamSynchronize(s));      // rec is rewritten for the next layout
    }
    for (int a = 0; a < 3 && !cb->loff_pad.empty(); ++a) {
        if (cb->loff_pad[a] < 0) continue;
        for (int i = 0; i < nbr; ++i) {
            rec[i].data_off = cb->loff_pad[3 * (size_t)i + a];
            layout_strides_padded(rec[i].dim, a, cb->storage == VR_F32 ? 4 : 2, rec[i].str);
        }
        CK(cudaMemcpyAsync(cb->d_tmpl, rec.data(), sizeof(DrawBrick) * nbr, cudaMemcpyHostToDevice, s));
        CK(launch_brick_build(cb->d_src, (int)cb->n[0], (int)cb->n[1], (int)cb->n[2], cb->d_tmpl, nbr, cb->d_bs,
                              cb->storage, cb->d_pool, d_exps, s));
        CK(cudaStreamSynchronize(s));
    }
    if (cb->storage != VR_F32) {
        std::vector<int> e(nbr);
        CK(cudaMemcpyAsync(e.data(), d_exps, sizeof(int) * nbr, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < nbr; ++i) cb->tmpl[i].exp2 = e[i];
    }
    if (cb->layouts & 8) return build_atlases(c, cb, s);
    free_atlases(cb);
    return VR_OK;
}

void free_cube(Cube *cb) {
    free_atlases(cb);
    if (cb->d_wstore) cudaFree(cb->d_wstore);
    if (cb->d_src) cudaFree(cb->d_src);
    if (cb->d_pool) cudaFree(cb->d_pool);
    if (cb->d_tmpl) cudaFree(cb->d_tmpl);
    if (cb->d_bs) cudaFree(cb->d_bs);
    delete cb;
}

}  // namespace

// =============================================================================================
// Rendering without allocation: a fixed device scratch array and a fixed host arena.
//
// Some callers cannot allocate device memory while they render: a process whose GPU memory is
// owned by another allocator or held to a fixed budget, or a frame loop that must not pay the
// device-wide synchronisation that cudaMalloc/cudaFree can cause.  vr_render_frame_noalloc
// serves them.  Its scratch (the staged work-list and the fragments) lives in the file-scope
// array below, reserved on every GPU that loads this library until the process exits.
// =============================================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;    // 64 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host arena the work-list is built in (static storage: no heap use on this path).  It is
// page-locked once (cudaHostRegister: the arena's own pages, nothing allocated), so the
// work-list upload is an asynchronous copy that waits for nothing queued before it.  The arena
// holds one work-list: a call first waits (bounded) until the previous call's upload has read
// it; the event recorded after each upload lives one per device (an event belongs to a device).
alignas(4096) unsigned char g_noalloc_host[kNoAllocScratchBytes];
std::mutex g_noalloc_mu;
bool g_noalloc_pinned = false;
constexpr int kNoAllocDevices = 256;
void *g_noalloc_dev[kNoAllocDevices] = {nullptr};              // device address, per device
cudaEvent_t g_noalloc_up[kNoAllocDevices] = {nullptr};         // "arena read", per device
int g_noalloc_last = -1;                                       // device of the last upload

// Device address of g_noalloc_scratch on the current device, and that device's upload event.
// In host code the symbol's name is only a stand-in; its address must be queried per device
// with that device current.
int noalloc_scratch(int device, unsigned char **ptr) {
    if (device < 0 || device >= kNoAllocDevices) return arg_fail("device ordinal out of range");
    if (!g_noalloc_pinned) {
        cudaError_t e = cudaHostRegister(g_noalloc_host, kNoAllocScratchBytes, cudaHostRegisterPortable);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostRegister(no-allocation host arena)");
        g_noalloc_pinned = true;
    }
    if (!g_noalloc_dev[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        e = cudaEventCreateWithFlags(&g_noalloc_up[device], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreateWithFlags");
        g_noalloc_dev[device] = p;
    }
    *ptr = static_cast<unsigned char *>(g_noalloc_dev[device]);
    return VR_OK;
}

// Waits until the last upload has read the host arena (60 s bound, VR_ERR_TIMEOUT).
int noalloc_arena_free() {
    if (g_noalloc_last < 0) return VR_OK;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t r = cudaEventQuery(g_noalloc_up[g_noalloc_last]);
        if (r == cudaSuccess) return VR_OK;
        if (r != cudaErrorNotReady) return cuda_fail(r, "cudaEventQuery");
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > 60.0)
            return fail(VR_ERR_TIMEOUT, "the previous work-list upload did not run within 60 s");
        std::this_thread::yield();
    }
}

struct StaticLayout {
    size_t off_lut, off_db, off_items, off_ts, off_tl, off_mask, bytes;
    int nd, nitems;
    long long frag_px;
};

// The work-list of build_worklist (same rectangles, culling, front-to-back order, bins),
// written straight into the static host arena.  Returns VR_ERR_ARG when it does not fit.
int build_worklist_static(vr_ctx *c, Cube *cb, unsigned char *arena, size_t cap, size_t frag_elem,
                          StaticLayout &L) {
    const Cam &cam = c->cam;
    const int W = cam.W, H = cam.H;
    const double R[9] = {cam.R[0], cam.R[1], cam.R[2], cam.R[3], cam.R[4], cam.R[5], cam.R[6], cam.R[7], cam.R[8]};
    const double t[3] = {cam.t[0], cam.t[1], cam.t[2]};
    int ecell[3] = {0, 0, 0}, dsign[3] = {1, 1, 1};
    if (cam.proj == VR_PERSP) {
        float e[3];
        eye_f32(cam, e);
        for (int a = 0; a < 3; ++a) {
            if (e[a] < 0.0f) ecell[a] = -1;
            else if (e[a] >= (float)cb->n[a]) ecell[a] = (int)cb->nb[a];
            else ecell[a] = std::min((int)(e[a] / (float)cb->B[a]), (int)cb->nb[a] - 1);
            while (ecell[a] > 0 && ecell[a] < cb->nb[a] && (float)((int64_t)ecell[a] * cb->B[a]) > e[a]) --ecell[a];
            while (ecell[a] + 1 < cb->nb[a] && (float)((int64_t)(ecell[a] + 1) * cb->B[a]) <= e[a]) ++ecell[a];
        }
    } else {
        for (int a = 0; a < 3; ++a) dsign[a] = (-cam.R[6 + a] >= 0.0f) ? 1 : -1;
    }
    const size_t nb = cb->tmpl.size();
    const int ntx = (W + kTile - 1) / kTile, nty = (H + kTile - 1) / kTile;
    const size_t ntiles = (size_t)ntx * nty;
    // scratch for candidates, sort keys and bin cursors at the top of the arena
    struct Key { long long key; int idx; };
    const size_t tmp_bytes = align_up(nb * sizeof(DrawBrick), 256) + align_up(nb * sizeof(Key), 256) +
                             align_up(ntiles * sizeof(int), 256);
    if (tmp_bytes >= cap) return arg_fail("frame does not fit the 64 MiB no-allocation scratch");
    unsigned char *tmp = arena + cap - tmp_bytes;
    DrawBrick *cand = reinterpret_cast<DrawBrick *>(tmp);
    Key *keys = reinterpret_cast<Key *>(tmp + align_up(nb * sizeof(DrawBrick), 256));
    int *cursor = reinterpret_cast<int *>(tmp + align_up(nb * sizeof(DrawBrick), 256) + align_up(nb * sizeof(Key), 256));
    int nc = 0;
    // the table has at most 4096 entries: its zero-opacity prefix fits on the stack
    int apre_buf[kMaxLut + 1];
    apre_buf[0] = 0;
    for (size_t i = 0; i < c->lut.size(); ++i) apre_buf[i + 1] = apre_buf[i] + (c->lut[i].w != 0.0f ? 1 : 0);
    // a partitioned cube draws its part (the equal split needs no heap; the balanced one does)
    const bool parted = cb->part_nlev > 0;
    const PartBox part = parted ? partition_box(c, cb) : PartBox{};
    for (size_t bi = 0; bi < nb; ++bi) {
        DrawBrick b = cb->tmpl[bi];
        if (parted && !in_part(part, cb, (int64_t)bi)) continue;
        if (!window_clip(c, cb, b, b.lo, b.hi)) continue;
        if (skip_brick(c, cb, bi, apre_buf)) continue;
        int x0 = 0, y0 = 0, x1 = W, y1 = H;
        bool cull = false;
        if (!c->full_rect) {
            double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
            int behind = 0, front = 0;
            for (int k = 0; k < 8; ++k) {
                double p[3] = {(k & 1) ? b.hi[0] : b.lo[0], (k & 2) ? b.hi[1] : b.lo[1], (k & 4) ? b.hi[2] : b.lo[2]};
                double e[3];
                for (int r = 0; r < 3; ++r) e[r] = R[3 * r] * p[0] + R[3 * r + 1] * p[1] + R[3 * r + 2] * p[2] + t[r];
                double sx, sy;
                if (cam.proj == VR_PERSP) {
                    if (e[2] > -1e-6) { ++behind; continue; }
                    ++front;
                    sx = e[0] / (-e[2]) / cam.th_w;
                    sy = e[1] / (-e[2]) / cam.th;
                } else {
                    if (e[2] > 0.0) ++behind; else ++front;
                    sx = e[0] / cam.half_w;
                    sy = e[1] / cam.half_h;
                }
                double px = (sx + 1.0) * 0.5 * W, py = (1.0 - sy) * 0.5 * H;
                mnx = std::min(mnx, px); mxx = std::max(mxx, px);
                mny = std::min(mny, py); mxy = std::max(mxy, py);
            }
            if (front == 0) {
                cull = true;
            } else if (cam.proj == VR_PERSP && behind > 0) {
                x0 = 0; y0 = 0; x1 = W; y1 = H;
            } else {
                // clamped to the frame in double first: the int conversion of an
                // out-of-range double is undefined
                x0 = (int)std::min((double)W, std::max(0.0, std::floor(mnx) - 1.0));
                y0 = (int)std::min((double)H, std::max(0.0, std::floor(mny) - 1.0));
                x1 = (int)std::max(0.0, std::min((double)W, std::ceil(mxx) + 1.0));
                y1 = (int)std::max(0.0, std::min((double)H, std::ceil(mxy) + 1.0));
                if (x1 <= x0 || y1 <= y0) cull = true;
            }
        }
        if (cull) continue;
        DrawBrick d = b;
        d.rect[0] = x0; d.rect[1] = y0; d.rect[2] = x1 - x0; d.rect[3] = y1 - y0;
        d.sampled = 0;
        int ci[3] = {(int)(b.brick % cb->nb[0]), (int)((b.brick / cb->nb[0]) % cb->nb[1]),
                     (int)(b.brick / (cb->nb[0] * cb->nb[1]))};
        long long key = 0;
        for (int a = 0; a < 3; ++a) {
            if (cam.proj == VR_PERSP) key += std::abs(ci[a] - ecell[a]);
            else key += dsign[a] > 0 ? ci[a] : (cb->nb[a] - 1 - ci[a]);
        }
        keys[nc] = Key{key, nc};
        cand[nc++] = d;
    }
    // (key, candidate index) is a total order: the same order as a stable sort by key
    std::sort(keys, keys + nc, [](const Key &a, const Key &b) { return a.key != b.key ? a.key < b.key : a.idx < b.idx; });
    const FrameLayout fl = frame_layout(c, cb);
    long long frag = 0, nitems = 0, nbin = 0;
    for (int i = 0; i < nc; ++i) {
        const DrawBrick &d = cand[keys[i].idx];
        frag += (long long)d.rect[2] * d.rect[3];
        nitems += (long long)((d.rect[2] + fl.tw - 1) / fl.tw) * ((d.rect[3] + fl.th - 1) / fl.th);
        nbin += (long long)((d.rect[0] + d.rect[2] - 1) / kTile - d.rect[0] / kTile + 1) *
                ((d.rect[1] + d.rect[3] - 1) / kTile - d.rect[1] / kTile + 1);
    }
    size_t off = 0;
    L.off_lut = off; off = align_up(off + sizeof(float4) * c->lut.size(), 256);
    L.off_db = off; off = align_up(off + sizeof(DrawBrick) * (size_t)nc, 256);
    L.off_items = off; off = align_up(off + sizeof(TileItem) * (size_t)nitems, 256);
    L.off_ts = off; off = align_up(off + sizeof(int) * (ntiles + 1), 256);
    L.off_tl = off; off = align_up(off + sizeof(int) * (size_t)nbin, 256);
    L.off_mask = off; off = align_up(off + c->chmask.size(), 256);
    L.bytes = off;
    L.nd = nc;
    L.nitems = (int)nitems;
    L.frag_px = frag;
    if (off + tmp_bytes > cap || off + (size_t)frag * frag_elem > cap) {
        g_last_error = "frame needs " + std::to_string(off + (size_t)frag * frag_elem) +
                       " bytes of scratch; the no-allocation limit is 64 MiB";
        return VR_ERR_ARG;
    }
    std::memcpy(arena + L.off_lut, c->lut.data(), sizeof(float4) * c->lut.size());
    if (!c->chmask.empty()) std::memcpy(arena + L.off_mask, c->chmask.data(), c->chmask.size());
    DrawBrick *db = reinterpret_cast<DrawBrick *>(arena + L.off_db);
    TileItem *items = reinterpret_cast<TileItem *>(arena + L.off_items);
    int *ts = reinterpret_cast<int *>(arena + L.off_ts);
    int *tl = reinterpret_cast<int *>(arena + L.off_tl);
    long long fo = 0, it = 0;
    for (int i = 0; i < nc; ++i) {
        DrawBrick d = cand[keys[i].idx];
        d.frag_off = fo;
        fo += (long long)d.rect[2] * d.rect[3];
        if (!cb->loff.empty()) d.data_off = cb->loff[3 * (size_t)d.brick + fl.layout];
        layout_strides(d.dim, fl.layout, d.str);
        d.pad_off = -1;
        if (!cb->loff_pad.empty() && cb->loff_pad[3 * (size_t)d.brick + fl.layout] >= 0) {
            d.pad_off = cb->loff_pad[3 * (size_t)d.brick + fl.layout];
            layout_strides_padded(d.dim, fl.layout, cb->storage == VR_F32 ? 4 : 2, d.pad_str);
        }
        const int tw = (d.rect[2] + fl.tw - 1) / fl.tw, th = (d.rect[3] + fl.th - 1) / fl.th;
        for (int ty = 0; ty < th; ++ty)
            for (int tx = 0; tx < tw; ++tx) items[it++] = TileItem{i, tx, ty};
        db[i] = d;
    }
    std::memset(ts, 0, sizeof(int) * (ntiles + 1));
    for (int i = 0; i < nc; ++i) {
        const DrawBrick &d = db[i];
        for (int ty = d.rect[1] / kTile; ty <= (d.rect[1] + d.rect[3] - 1) / kTile; ++ty)
            for (int tx = d.rect[0] / kTile; tx <= (d.rect[0] + d.rect[2] - 1) / kTile; ++tx)
                ts[(size_t)ty * ntx + tx + 1]++;
    }
    for (size_t i = 1; i <= ntiles; ++i) ts[i] += ts[i - 1];
    std::memcpy(cursor, ts, sizeof(int) * ntiles);
    for (int i = 0; i < nc; ++i) {
        const DrawBrick &d = db[i];
        for (int ty = d.rect[1] / kTile; ty <= (d.rect[1] + d.rect[3] - 1) / kTile; ++ty)
            for (int tx = d.rect[0] / kTile; tx <= (d.rect[0] + d.rect[2] - 1) / kTile; ++tx)
                tl[cursor[(size_t)ty * ntx + tx]++] = i;
    }
    return VR_OK;
}

}  // namespace

// =============================================================================================
// C ABI (the only symbols the library exports; everything else is built with hidden visibility)
// =============================================================================================
#pragma GCC visibility push(default)
extern "C" {

const char *vr_error_string(int status) {
    switch (status) {
        case VR_OK: return "VR_OK";
        case VR_ERR_ARG: return "VR_ERR_ARG: invalid argument";
        case VR_ERR_OOM: return "VR_ERR_OOM: out of memory";
        case VR_ERR_CUDA: return "VR_ERR_CUDA: CUDA runtime error";
        case VR_ERR_TIMEOUT: return "VR_ERR_TIMEOUT: bounded wait expired";
        case VR_ERR_STATE: return "VR_ERR_STATE: call out of order";
        case VR_ERR_NOT_FOUND: return "VR_ERR_NOT_FOUND: unknown cube id";
        case VR_ERR_UNSUPPORTED: return "VR_ERR_UNSUPPORTED: unsupported combination";
        case VR_ERR_IO: return "VR_ERR_IO: a brick source failed";
        default: return "unknown status";
    }
}

const char *vr_last_error_message(void) { return g_last_error.c_str(); }

static int vr_create_body(vr_ctx **out, int device, size_t cache_bytes);
int vr_create(vr_ctx **out, int device, size_t cache_bytes) {
    return abi_guard([&] { return vr_create_body(out, device, cache_bytes); });
}
static int vr_create_body(vr_ctx **out, int device, size_t cache_bytes) {
    if (!out) return arg_fail("null out");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return arg_fail("bad device");
    vr_ctx *c = new (std::nothrow) vr_ctx();
    if (!c) return VR_ERR_OOM;
    c->device = device;
    c->cache_bytes = cache_bytes;
    int rc = VR_OK;
    do {
        if ((e = cudaSetDevice(device)) != cudaSuccess) { rc = cuda_fail(e, "cudaSetDevice"); break; }
        if ((e = cudaStreamCreateWithFlags(&c->load_stream, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_fail(e, "stream"); break; }
        if ((e = cudaEventCreateWithFlags(&c->upload_done, cudaEventDisableTiming)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
        if ((e = cudaEventCreateWithFlags(&c->frame_done, cudaEventDisableTiming)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
        if ((e = cudaMalloc(&c->d_ctr, sizeof(Counters))) != cudaSuccess) { rc = cuda_fail(e, "counters"); break; }
        if ((e = cudaMemset(c->d_ctr, 0, sizeof(Counters))) != cudaSuccess) { rc = cuda_fail(e, "counters"); break; }
        if ((e = cudaMalloc(&c->d_mm, sizeof(unsigned int) * 2)) != cudaSuccess) { rc = cuda_fail(e, "minmax"); break; }
    } while (0);
    if (rc != VR_OK) { vr_destroy(c); return rc; }
    *out = c;
    return VR_OK;
}

static void vr_destroy_body(vr_ctx *c);
void vr_destroy(vr_ctx *c) {
    try {
        vr_destroy_body(c);
    } catch (...) {
    }
}
static void vr_destroy_body(vr_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    cache_destroy(c);
    for (auto &kv : c->cubes) free_cube(kv.second);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->d_stage.p) cudaFree(c->d_stage.p);
    if (c->d_frags.p) cudaFree(c->d_frags.p);
    if (c->d_gfrag.p) cudaFree(c->d_gfrag.p);
    if (c->d_gpart.p) cudaFree(c->d_gpart.p);
    if (c->d_gchunk.p) cudaFree(c->d_gchunk.p);
    if (c->d_gacc.p) cudaFree(c->d_gacc.p);
    if (c->d_out.p) cudaFree(c->d_out.p);
    if (c->d_ctr) cudaFree(c->d_ctr);
    if (c->d_mm) cudaFree(c->d_mm);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto &v : c->ev_pending) for (auto e : v) cudaEventDestroy(e);
    if (c->upload_done) cudaEventDestroy(c->upload_done);
    if (c->frame_done) cudaEventDestroy(c->frame_done);
    if (c->load_stream) cudaStreamDestroy(c->load_stream);
    delete c;
}

static int vr_load_cube_body(vr_ctx *c, const void *voxels, int dtype, int64_t nx, int64_t ny, int64_t nz, int where,
                 const int64_t *sub_origin, const int64_t *sub_extent, int *cube_id);
int vr_load_cube(vr_ctx *c, const void *voxels, int dtype, int64_t nx, int64_t ny, int64_t nz, int where,
                 const int64_t *sub_origin, const int64_t *sub_extent, int *cube_id) {
    return abi_guard([&] { return vr_load_cube_body(c, voxels, dtype, nx, ny, nz, where, sub_origin, sub_extent, cube_id); });
}
static int vr_load_cube_body(vr_ctx *c, const void *voxels, int dtype, int64_t nx, int64_t ny, int64_t nz, int where,
                 const int64_t *sub_origin, const int64_t *sub_extent, int *cube_id) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c || !voxels || !cube_id) return arg_fail("null argument");
    if (dtype != VR_F32) return arg_fail("dtype must be VR_F32");
    if (where != VR_HOST && where != VR_DEVICE) return arg_fail("bad location");
    if (nx <= 0 || ny <= 0 || nz <= 0) return arg_fail("non-positive size");
    if ((sub_origin == nullptr) != (sub_extent == nullptr)) return arg_fail("sub-cube needs origin and extent");
    int64_t org[3] = {0, 0, 0}, ext[3] = {nx, ny, nz}, full[3] = {nx, ny, nz};
    if (sub_origin) {
        for (int a = 0; a < 3; ++a) {
            org[a] = sub_origin[a];
            ext[a] = sub_extent[a];
            if (org[a] < 0 || ext[a] <= 0 || org[a] + ext[a] > full[a]) return arg_fail("sub-cube outside the array");
        }
    }
    if (ext[0] > (1 << 30) || ext[1] > (1 << 30) || ext[2] > (1 << 30)) return arg_fail("size too large");
    int rc = set_dev(c);
    if (rc) return rc;
    Cube *cb = new (std::nothrow) Cube();
    if (!cb) return VR_ERR_OOM;
    for (int a = 0; a < 3; ++a) cb->n[a] = ext[a];
    const size_t bytes = sizeof(float) * (size_t)ext[0] * ext[1] * ext[2];
    cudaError_t e = cudaMalloc(&cb->d_src, bytes);
    if (e != cudaSuccess) { delete cb; return cuda_fail(e, "cudaMalloc(cube)"); }
    cudaMemcpyKind kind = where == VR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // a device source is read after all work already queued on the device (the caller's
    // writes to it may still be in flight on any of its streams: the copy runs on the
    // library's own non-blocking stream, which orders after none of them)
    if (where == VR_DEVICE && (e = cudaDeviceSynchronize()) != cudaSuccess) {
        free_cube(cb);
        return cuda_fail(e, "cudaDeviceSynchronize (device cube source)");
    }
    // 3D copy of the box: rows of ext[0] floats
    cudaMemcpy3DParms p{};
    p.srcPtr = make_cudaPitchedPtr(const_cast<void *>(voxels), sizeof(float) * nx, nx, ny);
    p.srcPos = make_cudaPos(sizeof(float) * org[0], org[1], org[2]);
    p.dstPtr = make_cudaPitchedPtr(cb->d_src, sizeof(float) * ext[0], ext[0], ext[1]);
    p.extent = make_cudaExtent(sizeof(float) * ext[0], ext[1], ext[2]);
    p.kind = kind;
    e = cudaMemcpy3DAsync(&p, c->load_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->load_stream);
    if (e != cudaSuccess) { free_cube(cb); return cuda_fail(e, "cudaMemcpy3D(cube)"); }
    int id = c->next_id++;
    cb->id = id;
    c->cubes[id] = cb;
    *cube_id = id;
    return VR_OK;
}

static int vr_load_cube_procedural_body(vr_ctx *c, uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int *cube_id);
int vr_load_cube_procedural(vr_ctx *c, uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int *cube_id) {
    return abi_guard([&] { return vr_load_cube_procedural_body(c, seed, nx, ny, nz, cube_id); });
}
static int vr_load_cube_procedural_body(vr_ctx *c, uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int *cube_id) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c || !cube_id) return arg_fail("null argument");
    if (nx <= 0 || ny <= 0 || nz <= 0) return arg_fail("non-positive size");
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30)) return arg_fail("size too large");
    Cube *cb = new (std::nothrow) Cube();
    if (!cb) return VR_ERR_OOM;
    cb->n[0] = nx; cb->n[1] = ny; cb->n[2] = nz;
    cb->streamed = true;
    cb->proc_seed = seed;
    int id = c->next_id++;
    cb->id = id;
    c->cubes[id] = cb;
    *cube_id = id;
    return VR_OK;
}

static int vr_set_fault_injection_body(vr_ctx *c, int kind, int64_t after);
int vr_set_fault_injection(vr_ctx *c, int kind, int64_t after) {
    return abi_guard([&] { return vr_set_fault_injection_body(c, kind, after); });
}
static int vr_set_fault_injection_body(vr_ctx *c, int kind, int64_t after) {
    if (!c || kind < 0 || kind > 3) return arg_fail("bad fault injection");
    c->fault_kind = kind;
    c->fault_after = after;
    return VR_OK;
}

static int vr_update_cube_body(vr_ctx *c, int cube_id, const void *voxels, int where, void *stream);
int vr_update_cube(vr_ctx *c, int cube_id, const void *voxels, int where, void *stream) {
    return abi_guard([&] { return vr_update_cube_body(c, cube_id, voxels, where, stream); });
}
static int vr_update_cube_body(vr_ctx *c, int cube_id, const void *voxels, int where, void *stream) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c || !voxels) return arg_fail("null argument");
    if (where != VR_HOST && where != VR_DEVICE) return arg_fail("bad location");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (cb->streamed) return fail(VR_ERR_UNSUPPORTED, "streamed and compressed cubes have no resident voxels");
    int rc = set_dev(c);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(float) * (size_t)cb->n[0] * cb->n[1] * cb->n[2];
    if (c->frame_pending) CK(cudaStreamWaitEvent(s, c->frame_done, 0));
    CK(cudaMemcpyAsync(cb->d_src, voxels, bytes, where == VR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (cb->bricked) return build_bricks(c, cb, s);
    CK(cudaStreamSynchronize(s));
    return VR_OK;
}

static int vr_free_cube_body(vr_ctx *c, int cube_id);
int vr_free_cube(vr_ctx *c, int cube_id) {
    return abi_guard([&] { return vr_free_cube_body(c, cube_id); });
}
static int vr_free_cube_body(vr_ctx *c, int cube_id) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    set_dev(c);
    if (c->frame_pending) cudaEventSynchronize(c->frame_done);
    cache_forget_cube(c, cube_id);
    free_cube(cb);
    c->cubes.erase(cube_id);
    return VR_OK;
}

static int vr_compute_minmax_body(vr_ctx *c, int cube_id, float *vmin, float *vmax);
int vr_compute_minmax(vr_ctx *c, int cube_id, float *vmin, float *vmax) {
    return abi_guard([&] { return vr_compute_minmax_body(c, cube_id, vmin, vmax); });
}
static int vr_compute_minmax_body(vr_ctx *c, int cube_id, float *vmin, float *vmax) {
    if (!c || !vmin || !vmax) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (cb->streamed)
        return fail(VR_ERR_UNSUPPORTED, "min/max of a streamed or compressed cube would produce all of it");
    int rc = set_dev(c);
    if (rc) return rc;
    unsigned int init[2] = {0xffffffffu, 0u}, res[2];
    CK(cudaMemcpyAsync(c->d_mm, init, sizeof(init), cudaMemcpyHostToDevice, c->load_stream));
    CK(launch_minmax(cb->d_src, (long long)cb->n[0] * cb->n[1] * cb->n[2], c->d_mm, c->load_stream));
    CK(cudaMemcpyAsync(res, c->d_mm, sizeof(res), cudaMemcpyDeviceToHost, c->load_stream));
    CK(cudaStreamSynchronize(c->load_stream));
    auto dec = [](unsigned int e) {
        unsigned int b = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
        float f;
        std::memcpy(&f, &b, 4);
        return f;
    };
    *vmin = dec(res[0]);
    *vmax = dec(res[1]);
    return VR_OK;
}

static int vr_set_bricking_body(vr_ctx *c, int cube_id, int bx, int by, int bz, int ghost, int storage);
int vr_set_bricking(vr_ctx *c, int cube_id, int bx, int by, int bz, int ghost, int storage) {
    return abi_guard([&] { return vr_set_bricking_body(c, cube_id, bx, by, bz, ghost, storage); });
}
static int vr_set_bricking_body(vr_ctx *c, int cube_id, int bx, int by, int bz, int ghost, int storage) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (bx < 1 || by < 1 || bz < 1) return arg_fail("brick size < 1");
    if (ghost != 1) return arg_fail("ghost must be 1");
    if (storage != VR_F32 && storage != VR_F16 && storage != VR_BF16) return arg_fail("bad storage");
    if (cb->wavelet && storage != VR_F32) return fail(VR_ERR_UNSUPPORTED, "compressed cubes decode to FP32 bricks");
    int rc = set_dev(c);
    if (rc) return rc;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    const int B[3] = {bx, by, bz};
    int64_t nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (cb->n[a] + B[a] - 1) / B[a];
    const int64_t nbr = nb[0] * nb[1] * nb[2];
    if (nbr > (1 << 24)) return arg_fail("too many bricks");
    for (int a = 0; a < 3; ++a)
        if ((int64_t)std::min<int64_t>(B[a], cb->n[a]) + 2 * ghost > 65536) return arg_fail("brick too large");
    const size_t esz = storage == VR_F32 ? 4 : 2;
    std::vector<DrawBrick> t((size_t)nbr);
    size_t off = 0;  // elements
    for (int64_t bi = 0; bi < nbr; ++bi) {
        int64_t ci[3] = {bi % nb[0], (bi / nb[0]) % nb[1], bi / (nb[0] * nb[1])};
        DrawBrick &d = t[bi];
        std::memset(&d, 0, sizeof(d));
        for (int a = 0; a < 3; ++a) {
            int64_t lo = ci[a] * B[a], hi = std::min<int64_t>(lo + B[a], cb->n[a]);
            d.lo[a] = (float)lo;
            d.hi[a] = (float)hi;
            d.org[a] = (int)(lo - ghost);
            d.org_c[a] = (float)d.org[a] + 0.5f;
            d.dim[a] = (int)(hi - lo + 2 * ghost);
        }
        d.brick = (int)bi;
        d.pad_off = -1;
        const size_t elems = (size_t)d.dim[0] * d.dim[1] * d.dim[2];
        d.bytes = (long long)(elems * esz);
        layout_strides(d.dim, 0, d.str);
    }
    // the pool: one copy of every brick per kept layout (x-contiguous first)
    const int layouts = cb->streamed ? 1 : cb->layouts;
    std::vector<long long> loff((size_t)nbr * 3, -1);
    for (int a = 0; a < 3; ++a) {
        if (!(layouts & (1 << a))) continue;
        for (int64_t bi = 0; bi < nbr; ++bi) {
            loff[3 * bi + a] = (long long)off;
            off = align_up(off + (size_t)t[bi].dim[0] * t[bi].dim[1] * t[bi].dim[2], 64);
        }
    }
    // layout bit 4: padded copies of the kept linear layouts (resident cubes)
    std::vector<long long> loff_pad;
    if (!cb->streamed && (layouts & 16)) {
        loff_pad.assign((size_t)nbr * 3, -1);
        for (int a = 0; a < 3; ++a) {
            if (!(layouts & (1 << a))) continue;
            for (int64_t bi = 0; bi < nbr; ++bi) {
                int ps[3];
                loff_pad[3 * bi + a] = (long long)off;
                off = align_up(off + (size_t)layout_strides_padded(t[bi].dim, a, (int)esz, ps), 64);
            }
        }
    }
    for (int64_t bi = 0; bi < nbr; ++bi) t[bi].data_off = loff[3 * bi];
    if (cb->d_pool) { cudaFree(cb->d_pool); cb->d_pool = nullptr; }
    if (cb->d_tmpl) { cudaFree(cb->d_tmpl); cb->d_tmpl = nullptr; }
    cb->bricked = false;
    if (cb->streamed) {                // bricks are produced on demand into the cache
        cache_forget_cube(c, cube_id);    // (a cache with smaller slots is re-cut by the next frame)
        cb->tmpl = std::move(t);
        cb->loff.clear();
        cb->loff_pad.clear();
        for (int a = 0; a < 3; ++a) { cb->B[a] = B[a]; cb->nb[a] = nb[a]; }
        cb->ghost = ghost;
        cb->storage = storage;
        cb->bricked = true;
        return (cb->layouts & 8) ? cache_prepare_atlases(c, cb) : VR_OK;
    }
    CK(cudaMalloc(&cb->d_pool, std::max<size_t>(off * esz, 16)));
    cb->pool_bytes = off * esz;
    CK(cudaMalloc(&cb->d_tmpl, sizeof(DrawBrick) * nbr));
    CK(cudaMemcpy(cb->d_tmpl, t.data(), sizeof(DrawBrick) * nbr, cudaMemcpyHostToDevice));
    if (cb->d_bs) { cudaFree(cb->d_bs); cb->d_bs = nullptr; }
    CK(cudaMalloc(&cb->d_bs, sizeof(unsigned int) * 4 * nbr));
    cb->tmpl = std::move(t);
    cb->loff = std::move(loff);
    cb->loff_pad = std::move(loff_pad);
    for (int a = 0; a < 3; ++a) { cb->B[a] = B[a]; cb->nb[a] = nb[a]; }
    cb->ghost = ghost;
    cb->storage = storage;
    if (!cb->loff_pad.empty())          // row padding defined (it is copied, never sampled)
        CK(cudaMemsetAsync(cb->d_pool, 0, std::max<size_t>(off * esz, 16), c->load_stream));
    if ((rc = build_bricks(c, cb, c->load_stream)) != VR_OK) return rc;
    cb->bricked = true;
    return VR_OK;
}

static int vr_compress_cube_body(vr_ctx *c, int cube_id);
int vr_compress_cube(vr_ctx *c, int cube_id) {
    return abi_guard([&] { return vr_compress_cube_body(c, cube_id); });
}
static int vr_compress_cube_body(vr_ctx *c, int cube_id) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (cb->wavelet) return VR_OK;
    if (cb->streamed || !cb->d_src)
        return fail(VR_ERR_UNSUPPORTED, "only resident cubes (with their FP32 voxels) can be compressed");
    int rc;
    if ((rc = set_dev(c)) != VR_OK) return rc;
    size_t nb = 1;
    for (int a = 0; a < 3; ++a) nb *= (size_t)((cb->n[a] + 7) / 8);
    const size_t bytes = nb * (size_t)kWaveletRecordBytes;
    unsigned char *store = nullptr;
    CK(cudaMalloc(&store, bytes));
    cudaError_t e = launch_wavelet_encode(cb->d_src, (int)cb->n[0], (int)cb->n[1], (int)cb->n[2], store,
                                          c->load_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->load_stream);
    if (e != cudaSuccess) {
        cudaFree(store);
        return cuda_fail(e, "wavelet encode");
    }
    // the FP32 voxels, the brick pool and the atlases go; frames in flight may still read them
    CK(cudaDeviceSynchronize());
    free_atlases(cb);
    cudaFree(cb->d_src);
    cb->d_src = nullptr;
    if (cb->d_pool) { cudaFree(cb->d_pool); cb->d_pool = nullptr; }
    if (cb->d_tmpl) { cudaFree(cb->d_tmpl); cb->d_tmpl = nullptr; }
    if (cb->d_bs) { cudaFree(cb->d_bs); cb->d_bs = nullptr; }
    cb->pool_bytes = 0;
    cb->loff.clear();
    cb->loff_pad.clear();
    cb->vlo.clear();
    cb->vhi.clear();
    cb->d_wstore = store;
    cb->wstore_bytes = bytes;
    cb->wavelet = true;
    cb->streamed = true;
    cb->layouts = 1;
    if (!cb->bricked) return VR_OK;
    cb->bricked = false;                 // brick records for the cache, FP32 bricks
    return vr_set_bricking(c, cube_id, cb->B[0], cb->B[1], cb->B[2], cb->ghost, VR_F32);
}

static int vr_wavelet_store_body(vr_ctx *c, int cube_id, void *dst, size_t *bytes);
int vr_wavelet_store(vr_ctx *c, int cube_id, void *dst, size_t *bytes) {
    return abi_guard([&] { return vr_wavelet_store_body(c, cube_id, dst, bytes); });
}
static int vr_wavelet_store_body(vr_ctx *c, int cube_id, void *dst, size_t *bytes) {
    if (!c || !bytes) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (!cb->wavelet) return fail(VR_ERR_STATE, "cube is not compressed");
    if (!dst) {
        *bytes = cb->wstore_bytes;
        return VR_OK;
    }
    if (*bytes < cb->wstore_bytes) return arg_fail("destination smaller than the block store");
    int rc;
    if ((rc = set_dev(c)) != VR_OK) return rc;
    CK(cudaMemcpy(dst, cb->d_wstore, cb->wstore_bytes, cudaMemcpyDeviceToHost));
    *bytes = cb->wstore_bytes;
    return VR_OK;
}

static int vr_set_termination_body(vr_ctx *c, int mode);
int vr_set_termination(vr_ctx *c, int mode) {
    return abi_guard([&] { return vr_set_termination_body(c, mode); });
}
static int vr_set_termination_body(vr_ctx *c, int mode) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    if (mode != VR_TERM_SEGMENT && mode != VR_TERM_GLOBAL) return arg_fail("termination must be VR_TERM_SEGMENT or VR_TERM_GLOBAL");
    c->term = mode;
    return VR_OK;
}

static int vr_set_host_output_async_body(vr_ctx *c, int async);
int vr_set_host_output_async(vr_ctx *c, int async) {
    return abi_guard([&] { return vr_set_host_output_async_body(c, async); });
}
static int vr_set_host_output_async_body(vr_ctx *c, int async) {
    if (!c) return arg_fail("null ctx");
    if (async != 0 && async != 1) return arg_fail("async must be 0 or 1");
    c->async_host_out = async != 0;
    return VR_OK;
}

static int vr_set_brick_layouts_body(vr_ctx *c, int cube_id, int mask);
int vr_set_brick_layouts(vr_ctx *c, int cube_id, int mask) {
    return abi_guard([&] { return vr_set_brick_layouts_body(c, cube_id, mask); });
}
static int vr_set_brick_layouts_body(vr_ctx *c, int cube_id, int mask) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (mask < 1 || mask > 63 || !(mask & 1) || ((mask & 32) && !(mask & 8)))
        return arg_fail("layout mask must be 1..63, keep bit 0 (x contiguous), and set bit 3 with bit 5");
    if (cb->streamed && mask != 1 && mask != 9)
        return fail(VR_ERR_UNSUPPORTED, "streamed bricks are cached x-contiguous, with or without slot atlases (mask 1 or 9)");
    if (cb->layouts == mask) return VR_OK;
    cb->layouts = mask;
    if (!cb->bricked) return VR_OK;
    if (cb->streamed) {                // slot atlases: arrays made now, so that frames only pack
        if (!(mask & 8)) return VR_OK;
        int rc = set_dev(c);
        if (rc) return rc;
        return cache_prepare_atlases(c, cb);
    }
    return vr_set_bricking(c, cube_id, cb->B[0], cb->B[1], cb->B[2], cb->ghost, cb->storage);
}

// The table, camera and parameter setters count a change of the frame (state_gen, which the
// gradient calls compare before reusing a frame's fragments) only when the value changes:
// setting the same table, camera or parameters again leaves the last frame's fragments valid.
static int vr_set_transfer_function_body(vr_ctx *c, const float *rgba, int n, float vmin, float vmax);
int vr_set_transfer_function(vr_ctx *c, const float *rgba, int n, float vmin, float vmax) {
    return abi_guard([&] { return vr_set_transfer_function_body(c, rgba, n, vmin, vmax); });
}
static int vr_set_transfer_function_body(vr_ctx *c, const float *rgba, int n, float vmin, float vmax) {
    if (!c || !rgba) return arg_fail("null argument");
    if (n < 2 || n > kMaxLut) return arg_fail("table size must be 2..4096");
    if (!(vmax > vmin) || !std::isfinite(vmin) || !std::isfinite(vmax)) return arg_fail("need vmax > vmin");
    for (int i = 0; i < 4 * n; ++i)
        if (!std::isfinite(rgba[i])) return arg_fail("non-finite table entry");
    const bool same = c->tf_set && (int)c->lut.size() == n && c->vmin == vmin && c->vmax == vmax &&
                      std::memcmp(c->lut.data(), rgba, sizeof(float) * 4 * n) == 0;
    if (same) return VR_OK;
    c->state_gen++;
    c->lut.resize(n);
    std::memcpy(c->lut.data(), rgba, sizeof(float) * 4 * n);
    c->vmin = vmin;
    c->vmax = vmax;
    c->tf_set = true;
    return VR_OK;
}

static int vr_set_camera_body(vr_ctx *c, const float view[16], int proj, float param, int width, int height);
int vr_set_camera(vr_ctx *c, const float view[16], int proj, float param, int width, int height) {
    return abi_guard([&] { return vr_set_camera_body(c, view, proj, param, width, height); });
}
static int vr_set_camera_body(vr_ctx *c, const float view[16], int proj, float param, int width, int height) {
    if (!c || !view) return arg_fail("null argument");
    Cam cam;
    const int rc = make_cam(view, proj, param, width, height, cam);
    if (rc != VR_OK) return rc;
    if (c->cam_set && std::memcmp(&cam, &c->cam, sizeof(Cam)) == 0) return VR_OK;
    c->state_gen++;
    c->cam = cam;
    c->cam_set = true;
    return VR_OK;
}

static int vr_set_render_params_body(vr_ctx *c, int mode, float step, float tau);
int vr_set_render_params(vr_ctx *c, int mode, float step, float tau) {
    return abi_guard([&] { return vr_set_render_params_body(c, mode, step, tau); });
}
static int vr_set_render_params_body(vr_ctx *c, int mode, float step, float tau) {
    if (!c) return arg_fail("null ctx");
    if (mode != VR_DVR && mode != VR_MIP) return arg_fail("bad mode");
    if (!(step > 0.0f) || !std::isfinite(step)) return arg_fail("step must be > 0");
    if (!(tau > 0.0f) || std::isnan(tau)) return arg_fail("tau must be > 0");
    if (c->mode == mode && c->step == step && c->tau == tau) return VR_OK;
    c->state_gen++;
    c->mode = mode;
    c->step = step;
    c->tau = tau;
    return VR_OK;
}

static int vr_set_channel_mask_body(vr_ctx *c, const unsigned char *mask, int64_t n);
int vr_set_channel_mask(vr_ctx *c, const unsigned char *mask, int64_t n) {
    return abi_guard([&] { return vr_set_channel_mask_body(c, mask, n); });
}
static int vr_set_channel_mask_body(vr_ctx *c, const unsigned char *mask, int64_t n) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    if (!mask || n == 0) {
        c->chmask.clear();
        return VR_OK;
    }
    if (n < 0 || n > (1 << 30)) return arg_fail("bad channel count");
    c->chmask.assign(mask, mask + n);
    for (auto &m : c->chmask) m = m ? 1 : 0;
    return VR_OK;
}

static int vr_set_window_body(vr_ctx *c, const int64_t lo[3], const int64_t hi[3]);
int vr_set_window(vr_ctx *c, const int64_t lo[3], const int64_t hi[3]) {
    return abi_guard([&] { return vr_set_window_body(c, lo, hi); });
}
static int vr_set_window_body(vr_ctx *c, const int64_t lo[3], const int64_t hi[3]) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    if (!lo || !hi) {
        c->has_window = false;
        return VR_OK;
    }
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a])) return arg_fail("window must have hi > lo on every axis");
    for (int a = 0; a < 3; ++a) { c->win_lo[a] = lo[a]; c->win_hi[a] = hi[a]; }
    c->has_window = true;
    return VR_OK;
}

static int vr_set_timing_body(vr_ctx *c, int enable);
int vr_set_timing(vr_ctx *c, int enable) {
    return abi_guard([&] { return vr_set_timing_body(c, enable); });
}
static int vr_set_timing_body(vr_ctx *c, int enable) {
    if (!c) return arg_fail("null ctx");
    c->timing = enable != 0;
    return VR_OK;
}

static int vr_set_full_rect_body(vr_ctx *c, int full);
int vr_set_full_rect(vr_ctx *c, int full) {
    return abi_guard([&] { return vr_set_full_rect_body(c, full); });
}
static int vr_set_full_rect_body(vr_ctx *c, int full) {
    if (c) c->state_gen++;             // may change what a frame draws
    if (!c) return arg_fail("null ctx");
    c->full_rect = full != 0;
    return VR_OK;
}

}  // extern "C"

namespace vrh {

// The brick grid a global-termination frame walks: the cube's bricks, rays clipped to the cube
// or to the render window inside it.
__attribute__((visibility("hidden"))) MarchGrid march_grid(const vr_ctx *c, const Cube *cb) {
    MarchGrid g{};
    for (int a = 0; a < 3; ++a) {
        g.nb[a] = (int)cb->nb[a];
        g.B[a] = (float)cb->B[a];
        g.n[a] = (float)cb->n[a];
        g.invB[a] = 1.0f / g.B[a];
        g.clo[a] = 0.0f;
        g.chi[a] = (float)cb->n[a];
        if (c->has_window) {
            g.clo[a] = (float)std::max<int64_t>(c->win_lo[a], 0);
            g.chi[a] = (float)std::min<int64_t>(c->win_hi[a], cb->n[a]);
        }
    }
    return g;
}

// A DVR frame with global early termination: one launch in which every pixel's ray walks the
// cube's bricks front to back (k_raymarch), no fragments.  Stages the table, every brick's
// record (the frame's linear layout, atlas and skip flag) and the channel mask.
static int render_global(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s) {
    int rc;
    FrameConsts fc = make_consts(c, cb);
    FrameTiming tm(c);
    cudaEvent_t *ev = tm.ev;
    if (c->timing && (rc = timing_events(c, ev)) != VR_OK) return rc;
    const FrameLayout fl = frame_layout(c, cb);
    const size_t nb = cb->tmpl.size();
    std::vector<int> apre;
    alpha_prefix(c, apre);
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
    char *h = c->h_stage;
    std::memcpy(h + off_lut, c->lut.data(), sizeof(float4) * c->lut.size());
    DrawBrick *hb = reinterpret_cast<DrawBrick *>(h + off_b);
    int64_t drawn = 0;
    for (size_t i = 0; i < nb; ++i) {
        DrawBrick d = cb->tmpl[i];
        if (!cb->loff.empty()) d.data_off = cb->loff[3 * i + fl.layout];
        layout_strides(d.dim, fl.layout, d.str);
        d.skip = skip_brick(c, cb, i, apre.data()) ? 1 : 0;
        d.sampled = 0;
        drawn += d.skip ? 0 : 1;
        hb[i] = d;
    }
    if (!c->chmask.empty()) std::memcpy(h + off_mask, c->chmask.data(), c->chmask.size());
    const MarchGrid g = march_grid(c, cb);
    if (ev[0]) CK(cudaEventRecord(ev[0], s));
    CK(cudaMemcpyAsync(c->d_stage.p, h, off, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->upload_done, s));
    char *d = c->d_stage.p;
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
    if (empty) {                       // an empty window: a transparent frame
        CK(cudaMemsetAsync(dst, 0, opix * sizeof(float4), s));
    } else {
        CK(launch_raymarch(fc, reinterpret_cast<const float4 *>(d + off_lut), reinterpret_cast<DrawBrick *>(d + off_b),
                           g, cb->d_pool, reinterpret_cast<float4 *>(dst), c->d_ctr, s));
    }
    if (ev[2]) CK(cudaEventRecord(ev[2], s));
    if (ev[3]) CK(cudaEventRecord(ev[3], s));
    if (!direct) {
        CK(cudaMemcpyAsync(out, dst, opix * sizeof(float4),
                           out_where == VR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaEventRecord(c->frame_done, s));
    c->frame_pending = true;
    tm.queue();
    c->frames++;
    c->bricks_drawn += drawn;
    if (out_where == VR_HOST && !c->async_host_out) CK(cudaStreamSynchronize(s));
    return VR_OK;
}

// One frame of cube `cb` with the context's current table, camera and parameters.
__attribute__((visibility("hidden"))) int render_frame_impl(vr_ctx *c, Cube *cb, float *out, int out_where, cudaStream_t s) {
    int rc;
    if (cb->part_nlev > 0 && c->mode == VR_DVR && c->term == VR_TERM_GLOBAL)
        return fail(VR_ERR_UNSUPPORTED, "a partitioned cube's parts terminate per segment (VR_TERM_SEGMENT)");
    if (cb->streamed) {
        if (c->mode == VR_DVR && c->term == VR_TERM_GLOBAL) return render_streamed_global(c, cb, out, out_where, s);
        return render_streamed(c, cb, out, out_where, s);
    }
    if (c->mode == VR_DVR && c->term == VR_TERM_GLOBAL) return render_global(c, cb, out, out_where, s);
    FrameConsts fc = make_consts(c, cb);
    FrameTiming tm(c);
    cudaEvent_t *ev = tm.ev;
    if (c->timing && (rc = timing_events(c, ev)) != VR_OK) return rc;
    WorkList wl;
    if ((rc = stage_frame(c, cb, wl, s, ev[0])) != VR_OK) return rc;
    if (!c->chmask.empty()) fc.chmask = reinterpret_cast<const unsigned char *>(c->d_stage.p + wl.off_mask);
    const size_t opix = (size_t)fc.cam.W * fc.cam.H;
    const size_t fbytes = (size_t)wl.frag_px * (c->mode == VR_DVR ? sizeof(float4) : sizeof(float));
    c->frag_valid = false;
    if ((rc = ensure(c->d_frags, std::max<size_t>(fbytes, 16), c)) != VR_OK) return rc;
    const size_t ofl = opix * (c->mode == VR_DVR ? 4 : 1);
    float *dst = out;
    const bool direct = out_where == VR_DEVICE && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
    if (!direct) {
        if ((rc = ensure(c->d_out, ofl, c)) != VR_OK) return rc;
        dst = c->d_out.p;
    }
    char *d = c->d_stage.p;
    const float4 *d_lut = reinterpret_cast<const float4 *>(d + wl.off_lut);
    const DrawBrick *d_db = reinterpret_cast<const DrawBrick *>(d + wl.off_db);
    const TileItem *d_items = reinterpret_cast<const TileItem *>(d + wl.off_items);
    const int *d_ts = reinterpret_cast<const int *>(d + wl.off_ts);
    const int *d_tl = reinterpret_cast<const int *>(d + wl.off_tl);
    if (ev[1]) CK(cudaEventRecord(ev[1], s));
    CK(launch_raycast(fc, d_lut, d_db, d_items, (int)wl.items.size(), cb->d_pool, c->d_frags.p, c->d_ctr, s));
    if (c->mode == VR_DVR) {          // these fragments serve a backward pass of the same frame
        c->frag_valid = true;
        c->frag_cube = cb->id;
        c->frag_gen = c->state_gen;
    }
    if (ev[2]) CK(cudaEventRecord(ev[2], s));
    CK(launch_composite(fc, d_db, d_ts, d_tl, c->d_frags.p, dst, s));
    if (ev[3]) CK(cudaEventRecord(ev[3], s));
    if (!direct) {
        CK(cudaMemcpyAsync(out, dst, ofl * sizeof(float),
                           out_where == VR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaEventRecord(c->frame_done, s));
    c->frame_pending = true;
    tm.queue();
    c->frames++;
    c->fragments += wl.frag_px;
    c->bricks_drawn += (int64_t)wl.db.size();
    if (out_where == VR_HOST && !c->async_host_out) CK(cudaStreamSynchronize(s));
    return VR_OK;
}

}  // namespace vrh

extern "C" {

static int vr_render_frame_body(vr_ctx *c, int cube_id, float *out, int out_where, void *stream);
int vr_render_frame(vr_ctx *c, int cube_id, float *out, int out_where, void *stream) {
    return abi_guard([&] { return vr_render_frame_body(c, cube_id, out, out_where, stream); });
}
static int vr_render_frame_body(vr_ctx *c, int cube_id, float *out, int out_where, void *stream) {
    if (!c || !out) return arg_fail("null argument");
    if (out_where != VR_HOST && out_where != VR_DEVICE) return arg_fail("bad output location");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    int rc = check_ready(c, cb);
    if (rc) return rc;
    if ((rc = set_dev(c)) != VR_OK) return rc;
    return render_frame_impl(c, cb, out, out_where, static_cast<cudaStream_t>(stream));
}

static int vr_set_partition_body(vr_ctx *c, int cube_id, int nlevels, const int *counts, const int *index);
int vr_set_partition(vr_ctx *c, int cube_id, int nlevels, const int *counts, const int *index) {
    return abi_guard([&] { return vr_set_partition_body(c, cube_id, nlevels, counts, index); });
}
static int vr_set_partition_body(vr_ctx *c, int cube_id, int nlevels, const int *counts, const int *index) {
    if (!c) return arg_fail("null ctx");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (nlevels < 0 || nlevels > Cube::kMaxPartLevels) return arg_fail("nlevels must be 0..8");
    if (nlevels > 0 && (!counts || !index)) return arg_fail("null counts or index");
    for (int L = 0; L < nlevels; ++L)
        if (counts[L] < 1 || counts[L] > 65536 || index[L] < 0 || index[L] >= counts[L])
            return arg_fail("each level needs 1 <= counts <= 65536 and 0 <= index < counts");
    c->state_gen++;
    c->part_gen++;                    // a new part: the bricks' estimated costs still hold
    cb->part_nlev = nlevels;
    for (int L = 0; L < nlevels; ++L) { cb->part_counts[L] = counts[L]; cb->part_index[L] = index[L]; }
    return VR_OK;
}

static int vr_set_partition_balance_body(vr_ctx *c, int cube_id, int balanced);
int vr_set_partition_balance(vr_ctx *c, int cube_id, int balanced) {
    return abi_guard([&] { return vr_set_partition_balance_body(c, cube_id, balanced); });
}
static int vr_set_partition_balance_body(vr_ctx *c, int cube_id, int balanced) {
    if (!c) return arg_fail("null ctx");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (balanced != 0 && balanced != 1) return arg_fail("balanced must be 0 or 1");
    if (cb->part_balance != balanced) { c->state_gen++; c->part_gen++; }
    cb->part_balance = balanced;
    return VR_OK;
}

static int vr_get_partition_body(vr_ctx *c, int cube_id, int lo[3], int hi[3], int *axes);
int vr_get_partition(vr_ctx *c, int cube_id, int lo[3], int hi[3], int *axes) {
    return abi_guard([&] { return vr_get_partition_body(c, cube_id, lo, hi, axes); });
}
static int vr_get_partition_body(vr_ctx *c, int cube_id, int lo[3], int hi[3], int *axes) {
    if (!c || !lo || !hi) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (!cb->bricked) return fail(VR_ERR_STATE, "cube has no bricking");
    const PartBox p = partition_box(c, cb);
    for (int a = 0; a < 3; ++a) { lo[a] = p.lo[a]; hi[a] = p.hi[a]; }
    if (axes)
        for (int L = 0; L < cb->part_nlev; ++L) axes[L] = p.axis[L];
    return VR_OK;
}

static int vr_render_subimage_body(vr_ctx *c, int cube_id, float *out, int out_where, void *stream);
int vr_render_subimage(vr_ctx *c, int cube_id, float *out, int out_where, void *stream) {
    return abi_guard([&] { return vr_render_subimage_body(c, cube_id, out, out_where, stream); });
}
static int vr_render_subimage_body(vr_ctx *c, int cube_id, float *out, int out_where, void *stream) {
    if (!c || !out) return arg_fail("null argument");
    if (out_where != VR_HOST && out_where != VR_DEVICE) return arg_fail("bad output location");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    int rc = check_ready(c, cb);
    if (rc) return rc;
    if (c->mode == VR_DVR && c->term == VR_TERM_GLOBAL)
        return fail(VR_ERR_UNSUPPORTED, "sub-images composite per-segment fragments (VR_TERM_SEGMENT)");
    if ((rc = set_dev(c)) != VR_OK) return rc;
    c->subimage = true;
    rc = render_frame_impl(c, cb, out, out_where, static_cast<cudaStream_t>(stream));
    c->subimage = false;
    return rc;
}

static int vr_composite_subimages_body(vr_ctx *c, int cube_id, int level, int n, const float *subs, int row0, int rows,
                           int final_, float *out, void *stream);
int vr_composite_subimages(vr_ctx *c, int cube_id, int level, int n, const float *subs, int row0, int rows,
                           int final_, float *out, void *stream) {
    return abi_guard([&] { return vr_composite_subimages_body(c, cube_id, level, n, subs, row0, rows, final_, out, stream); });
}
static int vr_composite_subimages_body(vr_ctx *c, int cube_id, int level, int n, const float *subs, int row0, int rows,
                           int final_, float *out, void *stream) {
    if (!c || !subs || !out) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (!cb->bricked) return fail(VR_ERR_STATE, "cube has no bricking");
    if (!c->cam_set) return fail(VR_ERR_STATE, "no camera");
    if (level < 0 || level >= cb->part_nlev) return arg_fail("level outside the cube's partition");
    if (n != cb->part_counts[level]) return arg_fail("n must equal the partition's count at that level");
    if (row0 < 0 || rows < 0 || row0 + rows > c->cam.H) return arg_fail("rows outside the frame");
    if (reinterpret_cast<uintptr_t>(subs) % 16 != 0 || reinterpret_cast<uintptr_t>(out) % 16 != 0)
        return arg_fail("subs and out must be 16-byte aligned device memory");
    int rc = set_dev(c);
    if (rc) return rc;
    const PartBox p = partition_box(c, cb);
    FrameConsts fc{};
    fc.cam = c->cam;
    fc.mode = c->mode;
    fc.vmin = c->vmin;
    CK(launch_composite_parts(fc, p.axis[level], n, subs, row0, rows, final_ ? 1 : 0, out,
                              static_cast<cudaStream_t>(stream)));
    return VR_OK;
}

static int vr_render_backward_body(vr_ctx *c, int cube_id, const float *grad_out, float *grad_lut, float *grad_voxels,
                       void *stream);
int vr_render_backward(vr_ctx *c, int cube_id, const float *grad_out, float *grad_lut, float *grad_voxels,
                       void *stream) {
    return abi_guard([&] { return vr_render_backward_body(c, cube_id, grad_out, grad_lut, grad_voxels, stream); });
}
static int vr_render_backward_body(vr_ctx *c, int cube_id, const float *grad_out, float *grad_lut, float *grad_voxels,
                       void *stream) {
    if (!c || !grad_out || !grad_lut) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    int rc = backward_ready(c, cb);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(grad_out) % 16 != 0) return arg_fail("grad_out must be 16-byte aligned");
    if ((rc = set_dev(c)) != VR_OK) return rc;
    return backward_view(c, cb, grad_out, grad_lut, nullptr, false, grad_voxels, static_cast<cudaStream_t>(stream));
}

static int vr_render_backward_views_body(vr_ctx *c, int cube_id, int n_views, const vr_view *views, const float *grad_out,
                             float *grad_lut, float *grad_voxels, void *stream);
int vr_render_backward_views(vr_ctx *c, int cube_id, int n_views, const vr_view *views, const float *grad_out,
                             float *grad_lut, float *grad_voxels, void *stream) {
    return abi_guard([&] { return vr_render_backward_views_body(c, cube_id, n_views, views, grad_out, grad_lut, grad_voxels, stream); });
}
static int vr_render_backward_views_body(vr_ctx *c, int cube_id, int n_views, const vr_view *views, const float *grad_out,
                             float *grad_lut, float *grad_voxels, void *stream) {
    if (!c || !views || !grad_out || !grad_lut) return arg_fail("null argument");
    if (n_views < 1) return arg_fail("n_views must be >= 1");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    int rc = backward_ready(c, cb);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(grad_out) % 16 != 0) return arg_fail("grad_out must be 16-byte aligned");
    const int W = c->cam.W, H = c->cam.H;
    Cam probe;
    for (int v = 0; v < n_views; ++v)      // every view valid before any work is queued
        if ((rc = make_cam(views[v].view, views[v].proj, views[v].param, W, H, probe)) != VR_OK) return rc;
    if ((rc = set_dev(c)) != VR_OK) return rc;
    if ((rc = ensure(c->d_gacc, (size_t)4 * c->lut.size(), c)) != VR_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t per_view = (size_t)W * H * 4;
    // last view first: its fragments are usually the last frame's (render the batch, then
    // differentiate it), reused when the camera is unchanged
    for (int v = n_views - 1; v >= 0; --v) {
        Cam cam;
        make_cam(views[v].view, views[v].proj, views[v].param, W, H, cam);
        if (std::memcmp(&cam, &c->cam, sizeof(Cam)) != 0) {
            c->state_gen++;
            c->cam = cam;
        }
        rc = backward_view(c, cb, grad_out + (size_t)v * per_view, nullptr, c->d_gacc.p, v == n_views - 1,
                           grad_voxels, s);
        if (rc != VR_OK) return rc;
    }
    CK(launch_lut_grad_store(c->d_gacc.p, (int)c->lut.size(), grad_lut, s));
    CK(cudaEventRecord(c->frame_done, s));
    return VR_OK;
}

static int vr_get_stats_body(vr_ctx *c, vr_stats *st);
int vr_get_stats(vr_ctx *c, vr_stats *st) {
    return abi_guard([&] { return vr_get_stats_body(c, st); });
}
static int vr_get_stats_body(vr_ctx *c, vr_stats *st) {
    if (!c || !st) return arg_fail("null argument");
    int rc = set_dev(c);
    if (rc) return rc;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    if ((rc = collect_timing(c)) != VR_OK) return rc;
    Counters h{};
    CK(cudaMemcpy(&h, c->d_ctr, sizeof(h), cudaMemcpyDeviceToHost));
    std::memset(st, 0, sizeof(*st));
    st->frames = c->frames;
    st->samples = (int64_t)h.samples;
    st->fragments = c->fragments;
    st->bricks_drawn = c->bricks_drawn;
    st->bricks_sampled = (int64_t)h.bricks_sampled;
    st->brick_bytes_sampled = (int64_t)h.brick_bytes_sampled;
    st->ms_raycast = c->ms_raycast;
    st->ms_composite = c->ms_composite;
    st->ms_frame = c->ms_frame;
    st->timed_frames = c->timed_frames;
    st->kernel_errors = (int64_t)(h.pad & 0xffffffffull);
    cache_stats(c, st);
    return VR_OK;
}

static int vr_reset_stats_body(vr_ctx *c);
int vr_reset_stats(vr_ctx *c) {
    return abi_guard([&] { return vr_reset_stats_body(c); });
}
static int vr_reset_stats_body(vr_ctx *c) {
    if (!c) return arg_fail("null ctx");
    int rc = set_dev(c);
    if (rc) return rc;
    if (c->frame_pending) CK(cudaEventSynchronize(c->frame_done));
    if ((rc = collect_timing(c)) != VR_OK) return rc;
    CK(cudaMemset(c->d_ctr, 0, sizeof(Counters)));
    c->frames = c->fragments = c->bricks_drawn = c->timed_frames = 0;
    c->ms_raycast = c->ms_composite = c->ms_frame = 0;
    cache_reset_stats(c);
    return VR_OK;
}

static int vr_get_brick_grid_body(vr_ctx *c, int cube_id, int64_t nbricks[3], int *storage);
int vr_get_brick_grid(vr_ctx *c, int cube_id, int64_t nbricks[3], int *storage) {
    return abi_guard([&] { return vr_get_brick_grid_body(c, cube_id, nbricks, storage); });
}
static int vr_get_brick_grid_body(vr_ctx *c, int cube_id, int64_t nbricks[3], int *storage) {
    if (!c || !nbricks || !storage) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (!cb->bricked) return VR_ERR_STATE;
    for (int a = 0; a < 3; ++a) nbricks[a] = cb->nb[a];
    *storage = cb->storage;
    return VR_OK;
}

static int vr_get_brick_body(vr_ctx *c, int cube_id, int64_t brick, int dims[3], int org[3], int *exp2, void *data);
int vr_get_brick(vr_ctx *c, int cube_id, int64_t brick, int dims[3], int org[3], int *exp2, void *data) {
    return abi_guard([&] { return vr_get_brick_body(c, cube_id, brick, dims, org, exp2, data); });
}
static int vr_get_brick_body(vr_ctx *c, int cube_id, int64_t brick, int dims[3], int org[3], int *exp2, void *data) {
    if (!c || !dims || !org || !exp2) return arg_fail("null argument");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (!cb->bricked) return VR_ERR_STATE;
    if (brick < 0 || brick >= (int64_t)cb->tmpl.size()) return arg_fail("brick index out of range");
    int rc = set_dev(c);
    if (rc) return rc;
    const DrawBrick &b = cb->tmpl[brick];
    for (int a = 0; a < 3; ++a) { dims[a] = b.dim[a]; org[a] = b.org[a]; }
    *exp2 = b.exp2;
    if (cb->streamed) return data ? streamed_brick(cb, brick, data, exp2) : streamed_exp(cb, brick, exp2);
    if (data) {
        const size_t esz = cb->storage == VR_F32 ? 4 : 2;
        CK(cudaMemcpy(data, static_cast<char *>(cb->d_pool) + b.data_off * esz, (size_t)b.bytes, cudaMemcpyDeviceToHost));
    }
    return VR_OK;
}

// The no-allocation variant of vr_render_frame (see include/vrcube.h).
static int vr_render_frame_noalloc_body(vr_ctx *c, int cube_id, float *out, void *stream);
int vr_render_frame_noalloc(vr_ctx *c, int cube_id, float *out, void *stream) {
    return abi_guard([&] { return vr_render_frame_noalloc_body(c, cube_id, out, stream); });
}
static int vr_render_frame_noalloc_body(vr_ctx *c, int cube_id, float *out, void *stream) {
    if (!c || !out) return arg_fail("null argument");
    if (reinterpret_cast<uintptr_t>(out) % 16 != 0) return arg_fail("out must be 16-byte aligned device memory");
    Cube *cb = find_cube(c, cube_id);
    if (!cb) return VR_ERR_NOT_FOUND;
    if (cb->streamed) return fail(VR_ERR_UNSUPPORTED, "streamed cubes need the brick cache");
    if (c->mode == VR_DVR && c->term != VR_TERM_SEGMENT)
        return fail(VR_ERR_UNSUPPORTED, "the no-allocation path composites per-segment fragments (VR_TERM_SEGMENT)");
    if (cb->part_nlev > 0 && cb->part_balance)
        return fail(VR_ERR_UNSUPPORTED, "balanced partitions are computed on the heap; the no-allocation path takes equal ones");
    int rc = check_ready(c, cb);
    if (rc) return rc;
    if ((rc = set_dev(c)) != VR_OK) return rc;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned char *dev = nullptr;
    if ((rc = noalloc_scratch(c->device, &dev)) != VR_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FrameConsts fc = make_consts(c, cb);
    const size_t frag_elem = c->mode == VR_DVR ? sizeof(float4) : sizeof(float);
    StaticLayout L{};
    if ((rc = noalloc_arena_free()) != VR_OK) return rc;
    if ((rc = build_worklist_static(c, cb, g_noalloc_host, kNoAllocScratchBytes, frag_elem, L)) != VR_OK) return rc;
    // fragments follow the staged work-list; the kernel writes every fragment it later reads,
    // and the per-brick "sampled" flags arrive zeroed with the work-list, so nothing left over
    // from an earlier call is read
    CK(cudaMemcpyAsync(dev, g_noalloc_host, L.bytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(g_noalloc_up[c->device], s));
    g_noalloc_last = c->device;
    const float4 *d_lut = reinterpret_cast<const float4 *>(dev + L.off_lut);
    const DrawBrick *d_db = reinterpret_cast<const DrawBrick *>(dev + L.off_db);
    const TileItem *d_items = reinterpret_cast<const TileItem *>(dev + L.off_items);
    const int *d_ts = reinterpret_cast<const int *>(dev + L.off_ts);
    const int *d_tl = reinterpret_cast<const int *>(dev + L.off_tl);
    void *d_frags = dev + L.bytes;
    if (!c->chmask.empty()) fc.chmask = dev + L.off_mask;
    CK(launch_raycast(fc, d_lut, d_db, d_items, L.nitems, cb->d_pool, d_frags, c->d_ctr, s));
    CK(launch_composite(fc, d_db, d_ts, d_tl, d_frags, out, s));
    return VR_OK;
}

}  // extern "C"
#pragma GCC visibility pop
