// Continuous-batching server over the keyframe store (the `tm_server_*` calls of tm.h).
//
// Sec. V-F describes local mapping falling behind under a high keyframe rate: ORB-SLAM3
// keeps a fixed queue and skips stages when it is not empty.  Here keyframes are admitted as
// they arrive: a host thread packs the pending requests into a batch whenever one of
// `max_inflight_batches` stream slots is free and the store has room, ingests their
// keyframes (Sec. IV-B) and launches the batch's search + fusion as one persistent kernel,
// while earlier batches are still running on other streams.  A batch waits on the ingest of
// the batch before it, because its neighbours may have been ingested there.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "runtime.h"

using namespace tmap;

extern "C" double tm_now(void) {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

namespace {

struct Req {
    uint64_t ticket = 0, kf_id = 0;
    int n = 0;
    double Tcw[12];
    std::vector<uint8_t> desc, level, q_free, nbr_free;
    std::vector<float> xy, angle;
    std::vector<uint32_t> node;
    std::vector<uint64_t> nbrs;
    int n_mps = 0;
    std::vector<float> pos, normal, mind, maxd;
    std::vector<uint8_t> mdesc, skip;
    int n_fwd = 0;  // the new keyframe's own map points, fused into every neighbour
    std::vector<float> fpos, fnormal, fmind, fmaxd;
    std::vector<uint8_t> fdesc, fskip;
    // results
    bool done = false;
    tm_status status = TM_OK;
    std::vector<tm_match> matches;
    std::vector<int32_t> pair_offsets;
    std::vector<tm_fuse_match> fuse;
    std::vector<tm_fuse_match> fwd;
    std::vector<int32_t> fwd_offsets;
    std::vector<float> points;
    std::vector<uint8_t> point_ok;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Flight {
    BatchBuf B;
    IngestStage ingest;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr, ingested = nullptr;
    std::vector<Req *> reqs;
    std::vector<int> new_slots;
    bool busy = false;
    std::vector<tm_match> h_matches;
    std::vector<tm_fuse_match> h_fuse, h_fwd;
    std::vector<int32_t> h_pair_off, h_fuse_off, h_fwd_off;
    std::vector<float> h_points;
    std::vector<uint8_t> h_point_ok;
};

}  // namespace

struct tm_server {
    tm_ctx *ctx = nullptr;
    tm_server_config cfg{};
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    // keyframe id -> (keypoints, requests holding it) of the requests not yet taken: a
    // neighbour that is not stored yet may be the keyframe of an earlier request
    std::unordered_map<uint64_t, std::pair<int, int>> req_kf;
    std::vector<Flight> ring;
    std::deque<uint64_t> history;  // keyframes stored by this server, oldest first
    bool stopping = false;
    uint64_t next_ticket = 1;
    cudaEvent_t last_ingest = nullptr;
    tm_status thread_error = TM_OK;
    tm_server_stats stats{};  // under mu
};

extern "C" void tm_server_config_default(tm_server_config *c) {
    if (!c) return;
    c->max_batch_requests = 64;
    c->max_inflight_batches = 3;
    c->queue_capacity = 1 << 16;
    c->evict_after = 0;
    tm_search_params_default(&c->search);
    tm_fuse_params_default(&c->fuse);
    c->triangulate = 0;
    tm_triangulation_params_default(&c->tri);
}

namespace {

// Distribute the results of a finished flight to its requests.
void retire(tm_server *S, Flight &F) {
    Range range("tm_server retire (results to requests)");
    tm_ctx *c = S->ctx;
    tm_batch_result r{};
    r.matches = F.h_matches.data();
    r.match_cap = F.h_matches.size();
    r.fuse = F.h_fuse.data();
    r.fuse_cap = F.h_fuse.size();
    r.pair_offsets = F.h_pair_off.data();
    r.fuse_offsets = F.h_fuse_off.data();
    r.fwd = F.h_fwd.data();
    r.fwd_cap = F.h_fwd.size();
    r.fwd_offsets = F.h_fwd_off.data();
    const bool tri = S->cfg.triangulate != 0;
    if (tri) {
        r.points = F.h_points.data();
        r.point_ok = F.h_point_ok.data();
    }
    tm_status st = fetch_results(c, F.B, &r, F.stream);
    const double now = tm_now();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (int sl : F.B.slots) c->slots[sl].refs--;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t k = 0; k < F.reqs.size(); ++k) {
        Req *q = F.reqs[k];
        q->status = st;
        if (!st) {
            const int p0 = F.B.step_pair_begin[k], p1 = F.B.step_pair_begin[k + 1];
            const int base = F.h_pair_off[p0];
            q->matches.assign(F.h_matches.begin() + base, F.h_matches.begin() + F.h_pair_off[p1]);
            q->pair_offsets.resize(p1 - p0 + 1);
            for (int p = p0; p <= p1; ++p) q->pair_offsets[p - p0] = F.h_pair_off[p] - base;
            q->fuse.assign(F.h_fuse.begin() + F.h_fuse_off[k], F.h_fuse.begin() + F.h_fuse_off[k + 1]);
            const int fb = F.h_fwd_off[p0];
            q->fwd.assign(F.h_fwd.begin() + fb, F.h_fwd.begin() + F.h_fwd_off[p1]);
            q->fwd_offsets.resize(p1 - p0 + 1);
            for (int p = p0; p <= p1; ++p) q->fwd_offsets[p - p0] = F.h_fwd_off[p] - fb;
            if (tri) {
                const int me = F.h_pair_off[p1];
                q->points.assign(F.h_points.begin() + 3 * (size_t)base, F.h_points.begin() + 3 * (size_t)me);
                q->point_ok.assign(F.h_point_ok.begin() + base, F.h_point_ok.begin() + me);
            }
        }
        q->t_done = now;
        q->done = true;
        S->stats.completed++;
        if (st) S->stats.failed++;
    }
    F.reqs.clear();
    F.busy = false;
    S->cv_done.notify_all();
}

// Pack up to max_batch_requests pending requests into flight F and launch it.
// Returns false when nothing could be admitted (store full or queue empty).
bool admit(tm_server *S, Flight &F) {
    Range range("tm_server admit + launch");
    tm_ctx *c = S->ctx;
    std::vector<Req *> take;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        while (!S->pending.empty() && (int)take.size() < S->cfg.max_batch_requests) {
            take.push_back(S->pending.front());
            S->pending.pop_front();
        }
    }
    if (take.empty()) return false;
    const double now = tm_now();
    std::vector<Req *> ok;
    std::vector<tm_keyframe_view> views;
    std::vector<uint64_t> ids;
    std::vector<Req *> failed, deferred;
    int64_t evicted = 0;
    int slots_in_use = 0;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        cudaSetDevice(c->device);
        // admission by store memory: evict the oldest keyframes of the stream if asked to
        auto evict = [&]() {
            while (S->cfg.evict_after > 0 && (int)S->history.size() > S->cfg.evict_after) {
                const uint64_t old = S->history.front();
                auto it = c->ids.find(old);
                if (it != c->ids.end()) {
                    if (c->slots[it->second].refs > 0) break;
                    c->free_slots.push_back(it->second);
                    c->ids.erase(it);
                    ++evicted;
                }
                S->history.pop_front();
            }
        };
        evict();
        std::vector<int> slots;
        std::unordered_map<uint64_t, int> batch_ids;
        for (Req *q : take) {
            // once a request waits for store memory, the later ones wait too (arrival order):
            // they are checked when they are taken, so that a neighbour that is a waiting
            // request's keyframe is not taken for a missing one
            if (!deferred.empty()) {
                deferred.push_back(q);
                continue;
            }
            tm_keyframe_view v{};
            v.n = q->n;
            v.desc = q->desc.data();
            v.xy = q->xy.data();
            v.angle = q->angle.data();
            v.level = q->level.data();
            v.node = q->node.data();
            memcpy(v.Tcw, q->Tcw, sizeof v.Tcw);
            tm_status st = validate_view(c, v);
            if (!st && (c->ids.count(q->kf_id) || batch_ids.count(q->kf_id))) st = TM_ERR_EXISTS;
            size_t nbr_kp = 0;  // the neighbours' keypoints: the length nbr_free must have
            if (!st)
                for (uint64_t nb : q->nbrs) {
                    auto it = c->ids.find(nb);
                    if (it != c->ids.end()) {
                        nbr_kp += (size_t)c->slots[it->second].n;
                    } else {
                        auto bt = batch_ids.find(nb);
                        if (bt == batch_ids.end()) { st = TM_ERR_NOT_FOUND; break; }
                        nbr_kp += (size_t)views[(size_t)bt->second].n;
                    }
                }
            if (!st && !q->nbr_free.empty() && q->nbr_free.size() != nbr_kp) st = TM_ERR_INVALID_ARG;
            if (st) {
                q->status = st;
                failed.push_back(q);
                continue;
            }
            // admission by memory: a store slot for the new keyframe
            std::vector<int> got;
            const tm_status a = alloc_slots_locked(c, 1, got);
            if (!a) slots.push_back(got[0]);
            if (a) {
                deferred.push_back(q);
                continue;
            }
            batch_ids[q->kf_id] = (int)ok.size();
            ok.push_back(q);
            views.push_back(v);
            ids.push_back(q->kf_id);
        }
        if (!ok.empty()) {
            // ingest after the previous batch's ingest (neighbours may come from it)
            if (S->last_ingest) cudaStreamWaitEvent(F.stream, S->last_ingest, 0);
            tm_status st = enqueue_ingest(c, F.ingest, (int)ok.size(), views.data(), slots.data(), F.stream);
            if (st) {
                for (int sl : slots) c->free_slots.push_back(sl);
                for (Req *q : ok) { q->status = st; failed.push_back(q); }
                ok.clear();
            } else {
                for (size_t k = 0; k < ok.size(); ++k) {
                    Slot &sl = c->slots[slots[k]];
                    sl.n = views[k].n;
                    sl.refs = 0;
                    sl.id = ids[k];
                    c->ids[ids[k]] = slots[k];
                    S->history.push_back(ids[k]);
                }
                cudaEventRecord(F.ingested, F.stream);
                S->last_ingest = F.ingested;
            }
        }
        if (!ok.empty()) {
            // one batch: masks and map points of all requests concatenated
            std::vector<tm_step> steps(ok.size());
            std::vector<uint8_t> masks;
            size_t nm = 0;
            for (Req *q : ok) nm += (size_t)q->n_mps + (size_t)q->n_fwd;
            std::vector<float> pos(3 * nm), normal(3 * nm), mind(nm), maxd(nm);
            std::vector<uint8_t> mdesc(32 * nm), skip(nm);
            size_t mo = 0;
            bool any_skip = false;
            for (size_t k = 0; k < ok.size(); ++k) {
                Req *q = ok[k];
                tm_step &s = steps[k];
                s.kf_id = q->kf_id;
                s.nbr_ids = q->nbrs.data();
                s.n_nbrs = (int)q->nbrs.size();
                s.q_free_off = -1;
                s.nbr_free_off = -1;
                if (!q->q_free.empty()) {
                    s.q_free_off = (int64_t)masks.size();
                    masks.insert(masks.end(), q->q_free.begin(), q->q_free.end());
                }
                if (!q->nbr_free.empty()) {
                    s.nbr_free_off = (int64_t)masks.size();
                    masks.insert(masks.end(), q->nbr_free.begin(), q->nbr_free.end());
                }
                s.mp_begin = (int)mo;
                s.mp_count = q->n_mps;
                if (q->n_mps) {
                    memcpy(&pos[3 * mo], q->pos.data(), 12 * (size_t)q->n_mps);
                    memcpy(&normal[3 * mo], q->normal.data(), 12 * (size_t)q->n_mps);
                    memcpy(&mind[mo], q->mind.data(), 4 * (size_t)q->n_mps);
                    memcpy(&maxd[mo], q->maxd.data(), 4 * (size_t)q->n_mps);
                    memcpy(&mdesc[32 * mo], q->mdesc.data(), 32 * (size_t)q->n_mps);
                    if (!q->skip.empty()) {
                        memcpy(&skip[mo], q->skip.data(), (size_t)q->n_mps);
                        any_skip = true;
                    }
                }
                mo += (size_t)q->n_mps;
                // forward fusion: the request's own map points, after its backward ones (their
                // skip flags stay 0: the per-neighbour skip bytes decide)
                s.fwd_mp_begin = (int)mo;
                s.fwd_mp_count = q->n_fwd;
                s.fwd_skip_off = -1;
                if (q->n_fwd) {
                    const size_t f = (size_t)q->n_fwd;
                    memcpy(&pos[3 * mo], q->fpos.data(), 12 * f);
                    memcpy(&normal[3 * mo], q->fnormal.data(), 12 * f);
                    memcpy(&mind[mo], q->fmind.data(), 4 * f);
                    memcpy(&maxd[mo], q->fmaxd.data(), 4 * f);
                    memcpy(&mdesc[32 * mo], q->fdesc.data(), 32 * f);
                    if (!q->fskip.empty()) {
                        s.fwd_skip_off = (int64_t)masks.size();
                        masks.insert(masks.end(), q->fskip.begin(), q->fskip.end());
                    }
                }
                mo += (size_t)q->n_fwd;
            }
            tm_batch_inputs in{};
            in.masks = masks.empty() ? nullptr : masks.data();
            in.mask_bytes = masks.size();
            in.mps.n = (int)nm;
            in.mps.pos = pos.data();
            in.mps.normal = normal.data();
            in.mps.desc = mdesc.data();
            in.mps.min_dist = mind.data();
            in.mps.max_dist = maxd.data();
            in.mps.skip = any_skip ? skip.data() : nullptr;
            in.tri = S->cfg.triangulate ? &S->cfg.tri : nullptr;
            tm_status st = prepare_batch(c, F.B, steps.data(), (int)steps.size(), &in, S->cfg.search,
                                         S->cfg.fuse, F.stream);
            if (!st) {
                int th = default_threads(c, F.B), ln = c->def_lanes;
                if (S->cfg.search.lanes_per_query) ln = S->cfg.search.lanes_per_query;
                // the last tuned plan's launch choices (served requests are not measured)
                F.B.knobs = c->last_staged == 1 ? c->last_knobs : Knobs{};
                st = S->cfg.search.mode == TM_MODE_PER_PAIR ? enqueue_plain(c, F.B, ln, F.stream)
                                                            : enqueue_fused(c, F.B, th, ln, F.stream);
            }
            // host inputs of the copies above are pageable vectors: the copies have been
            // staged by the time cudaMemcpyAsync returned, so they may go out of scope.
            if (st) {
                for (Req *q : ok) { q->status = st; failed.push_back(q); }
                ok.clear();
            } else {
                for (int sl : F.B.slots) c->slots[sl].refs++;
                cudaEventRecord(F.done, F.stream);
            }
        }
        slots_in_use = (int)(c->slots.size() - c->free_slots.size());
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) S->pending.push_front(*it);
        for (Req *q : failed) {
            q->done = true;
            q->t_admit = q->t_done = tm_now();
        }
        for (Req *q : ok) q->t_admit = now;
        if (!failed.empty()) S->cv_done.notify_all();
        tm_server_stats &sx = S->stats;
        sx.admitted += (int64_t)ok.size();
        sx.failed += (int64_t)failed.size();
        sx.completed += (int64_t)failed.size();
        sx.deferrals += deferred.empty() ? 0 : 1;
        sx.evicted += evicted;
        sx.batches += ok.empty() ? 0 : 1;
        sx.peak_store_slots = std::max(sx.peak_store_slots, slots_in_use);
        if (!ok.empty()) {
            int infl = 1;
            for (Flight &G : S->ring) infl += (&G != &F && G.busy) ? 1 : 0;
            sx.peak_inflight = std::max(sx.peak_inflight, infl);
        }
    }
    if (ok.empty()) return !failed.empty();
    F.reqs = ok;
    F.busy = true;
    size_t pad = std::max<size_t>(1, F.B.total_pad);
    F.h_matches.resize(pad);
    F.h_fuse.resize(pad);
    F.h_pair_off.resize(F.B.n_pairs + 1);
    F.h_fuse_off.resize(F.B.n_steps + 1);
    F.h_fwd.resize(pad);
    F.h_fwd_off.resize(F.B.n_pairs + 1);
    if (S->cfg.triangulate) {
        F.h_points.resize(3 * pad);
        F.h_point_ok.resize(pad);
    }
    return true;
}

void server_loop(tm_server *S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        bool progressed = false;
        for (Flight &F : S->ring)
            if (F.busy && cudaEventQuery(F.done) == cudaSuccess) {
                retire(S, F);
                progressed = true;
            }
        for (Flight &F : S->ring)
            if (!F.busy) {
                if (admit(S, F)) progressed = true;
                break;
            }
        bool busy = false;
        for (Flight &F : S->ring) busy |= F.busy;
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stopping && !busy && !progressed) {
            // whatever still waits for store memory cannot be admitted any more
            for (Req *q : S->pending) {
                q->status = TM_ERR_NO_MEMORY;
                q->done = true;
                q->t_done = tm_now();
                S->stats.completed++;
                S->stats.failed++;
            }
            S->pending.clear();
            S->cv_done.notify_all();
            break;
        }
        if (!progressed) {
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
}

}  // namespace

extern "C" tm_status tm_server_start(tm_ctx *c, const tm_server_config *cfg, tm_server **out) {
    if (!c || !out) return fail(TM_ERR_INVALID_ARG, "tm_server_start: null argument");
    tm_server_config d;
    tm_server_config_default(&d);
    if (cfg) d = *cfg;
    if (d.max_batch_requests < 1 || d.max_inflight_batches < 1 || d.queue_capacity < 1)
        return fail(TM_ERR_INVALID_ARG, "tm_server_start: bad configuration");
    cudaSetDevice(c->device);
    tm_server *S = new tm_server();
    S->ctx = c;
    S->cfg = d;
    S->ring.resize(d.max_inflight_batches);
    for (Flight &F : S->ring) {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&F.stream, cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&F.done, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&F.ingested, cudaEventDisableTiming))) {
            delete S;
            return cuda_fail(e, "server streams");
        }
    }
    S->th = std::thread(server_loop, S);
    *out = S;
    return TM_OK;
}

extern "C" tm_status tm_server_submit(tm_server *S, const tm_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return fail(TM_ERR_INVALID_ARG, "tm_server_submit: null argument");
    const tm_keyframe_view &v = r->kf;
    if (v.n < 0 || v.n > S->ctx->cap) return fail(TM_ERR_INVALID_ARG, "tm_server_submit: bad keypoint count");
    if (v.n > 0 && (!v.desc || !v.xy || !v.angle || !v.level || !v.node))
        return fail(TM_ERR_INVALID_ARG, "tm_server_submit: null keyframe array");
    if (r->n_nbrs < 0 || (r->n_nbrs > 0 && !r->nbr_ids)) return fail(TM_ERR_INVALID_ARG, "tm_server_submit: bad neighbours");
    const tm_mappoint_view &m = r->mps, &fm = r->fwd_mps;
    if (m.n < 0 || (m.n > 0 && (!m.pos || !m.normal || !m.desc || !m.min_dist || !m.max_dist)))
        return fail(TM_ERR_INVALID_ARG, "tm_server_submit: bad map points");
    if (fm.n < 0 || (fm.n > 0 && (!fm.pos || !fm.normal || !fm.desc || !fm.min_dist || !fm.max_dist)))
        return fail(TM_ERR_INVALID_ARG, "tm_server_submit: bad forward map points");
    auto q = std::make_unique<Req>();
    q->kf_id = r->kf_id;
    q->n = v.n;
    memcpy(q->Tcw, v.Tcw, sizeof q->Tcw);
    const size_t n = (size_t)v.n;
    q->desc.assign(v.desc, v.desc + 32 * n);
    q->xy.assign(v.xy, v.xy + 2 * n);
    q->angle.assign(v.angle, v.angle + n);
    q->level.assign(v.level, v.level + n);
    q->node.assign(v.node, v.node + n);
    q->nbrs.assign(r->nbr_ids, r->nbr_ids + r->n_nbrs);
    if (r->q_free) q->q_free.assign(r->q_free, r->q_free + n);
    if (r->nbr_free && r->nbr_free_bytes) {
        q->nbr_free.assign(r->nbr_free, r->nbr_free + r->nbr_free_bytes);
    } else if (r->nbr_free) {
        // the concatenation length (sum of the neighbours' keypoint counts) from their sizes:
        // stored keyframes, or the keyframes of earlier requests
        size_t tot = 0;
        {
            std::lock_guard<std::mutex> lk(S->ctx->mu);
            for (uint64_t nb : q->nbrs) {
                auto it = S->ctx->ids.find(nb);
                if (it != S->ctx->ids.end()) tot += (size_t)S->ctx->slots[it->second].n;
                else {
                    std::lock_guard<std::mutex> lk2(S->mu);
                    auto rk = S->req_kf.find(nb);
                    if (rk == S->req_kf.end()) return fail(TM_ERR_NOT_FOUND, "neighbour %llu unknown", (unsigned long long)nb);
                    tot += (size_t)rk->second.first;
                }
            }
        }
        q->nbr_free.assign(r->nbr_free, r->nbr_free + tot);
    }
    q->n_mps = m.n;
    const size_t nm = (size_t)m.n;
    if (nm) {
        q->pos.assign(m.pos, m.pos + 3 * nm);
        q->normal.assign(m.normal, m.normal + 3 * nm);
        q->mdesc.assign(m.desc, m.desc + 32 * nm);
        q->mind.assign(m.min_dist, m.min_dist + nm);
        q->maxd.assign(m.max_dist, m.max_dist + nm);
        if (m.skip) q->skip.assign(m.skip, m.skip + nm);
    }
    q->n_fwd = fm.n;
    const size_t nf = (size_t)fm.n;
    if (nf) {
        q->fpos.assign(fm.pos, fm.pos + 3 * nf);
        q->fnormal.assign(fm.normal, fm.normal + 3 * nf);
        q->fdesc.assign(fm.desc, fm.desc + 32 * nf);
        q->fmind.assign(fm.min_dist, fm.min_dist + nf);
        q->fmaxd.assign(fm.max_dist, fm.max_dist + nf);
        if (r->fwd_skip) q->fskip.assign(r->fwd_skip, r->fwd_skip + nf * (size_t)r->n_nbrs);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->pending.size() >= S->cfg.queue_capacity) return fail(TM_ERR_BUSY, "server queue full");
    if (S->stopping) return fail(TM_ERR_BUSY, "server stopping");
    q->ticket = S->next_ticket++;
    q->t_submit = tm_now();
    *ticket = q->ticket;
    S->pending.push_back(q.get());
    {
        auto &e = S->req_kf[q->kf_id];
        e.first = q->n;
        ++e.second;
    }
    S->reqs[q->ticket] = std::move(q);
    S->stats.submitted++;
    S->stats.peak_pending = std::max(S->stats.peak_pending, (int32_t)S->pending.size());
    S->cv_work.notify_one();
    return TM_OK;
}

extern "C" tm_status tm_server_get_stats(tm_server *S, tm_server_stats *out) {
    if (!S || !out) return fail(TM_ERR_INVALID_ARG, "tm_server_get_stats: null argument");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        *out = S->stats;
    }
    tm_ctx *c = S->ctx;
    out->store_slot_limit = c->budget ? (int32_t)std::min<size_t>(c->budget / c->slot_bytes, INT32_MAX) : -1;
    return TM_OK;
}

extern "C" tm_status tm_server_poll(tm_server *S, uint64_t ticket, double timeout_s, tm_request_info *info) {
    if (!S || !info) return fail(TM_ERR_INVALID_ARG, "tm_server_poll: null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(TM_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second.get();
    if (!q->done && timeout_s > 0)
        S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return q->done; });
    info->done = q->done ? 1 : 0;
    info->status = q->status;
    info->n_matches = (int32_t)q->matches.size();
    info->n_fuse = (int32_t)q->fuse.size();
    info->n_fwd = (int32_t)q->fwd.size();
    info->t_submit = q->t_submit;
    info->t_admit = q->t_admit;
    info->t_done = q->t_done;
    if (!q->done && timeout_s > 0) return fail(TM_ERR_TIMEOUT, "request %llu not done", (unsigned long long)ticket);
    return TM_OK;
}

extern "C" tm_status tm_server_take(tm_server *S, uint64_t ticket, tm_match *matches,
                                    int32_t *pair_offsets, tm_fuse_match *fuse) {
    return tm_server_take_ex(S, ticket, matches, pair_offsets, fuse, nullptr, nullptr, nullptr, nullptr);
}

extern "C" tm_status tm_server_take_ex(tm_server *S, uint64_t ticket, tm_match *matches,
                                       int32_t *pair_offsets, tm_fuse_match *fuse, tm_fuse_match *fwd,
                                       int32_t *fwd_offsets, float *points, uint8_t *point_ok) {
    if (!S) return fail(TM_ERR_INVALID_ARG, "tm_server_take: null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(TM_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second.get();
    if (!q->done) return fail(TM_ERR_BUSY, "request %llu not done", (unsigned long long)ticket);
    auto forget = [&]() {
        auto rk = S->req_kf.find(q->kf_id);
        if (rk != S->req_kf.end() && --rk->second.second <= 0) S->req_kf.erase(rk);
        S->reqs.erase(it);
    };
    if (q->status) {
        tm_status s = q->status;
        forget();
        return fail(s, "request failed with status %d", s);
    }
    if (matches && !q->matches.empty()) memcpy(matches, q->matches.data(), q->matches.size() * sizeof(tm_match));
    if (pair_offsets) memcpy(pair_offsets, q->pair_offsets.data(), q->pair_offsets.size() * sizeof(int32_t));
    if (fuse && !q->fuse.empty()) memcpy(fuse, q->fuse.data(), q->fuse.size() * sizeof(tm_fuse_match));
    if (fwd && !q->fwd.empty()) memcpy(fwd, q->fwd.data(), q->fwd.size() * sizeof(tm_fuse_match));
    if (fwd_offsets && !q->fwd_offsets.empty())
        memcpy(fwd_offsets, q->fwd_offsets.data(), q->fwd_offsets.size() * sizeof(int32_t));
    if (points && !q->points.empty()) memcpy(points, q->points.data(), q->points.size() * sizeof(float));
    if (point_ok && !q->point_ok.empty()) memcpy(point_ok, q->point_ok.data(), q->point_ok.size());
    forget();
    return TM_OK;
}

extern "C" tm_status tm_server_stop(tm_server *S) {
    if (!S) return fail(TM_ERR_INVALID_ARG, "tm_server_stop: null server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->ctx->device);
    for (Flight &F : S->ring) {
        if (F.stream) cudaStreamSynchronize(F.stream);
        F.B.release();
        F.ingest.release();
        if (F.done) cudaEventDestroy(F.done);
        if (F.ingested) cudaEventDestroy(F.ingested);
        if (F.stream) cudaStreamDestroy(F.stream);
    }
    delete S;
    return TM_OK;
}
