// Internal host-side state of the library (context, store, batches).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "kernels.h"
#include "layout.cuh"
#include "tm.h"

namespace tmap {

// Largest entry list of the entry form (entries of 8 bytes: 512 MB).
constexpr long long kEntryCapMax = 1LL << 26;

// A host-side NVTX range over a scope: the library's calls and their stages appear on the
// timeline of a profiler attached to the process (with none attached a push costs a few ns).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    unsigned generation = 0;
    cudaError_t reserve(size_t n);  // grows (contents not kept)
    void release();
};

struct PinBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n);
    void release();
};

struct Slot {
    unsigned char *ptr = nullptr;
    int n = 0;
    int refs = 0;
    uint64_t id = 0;
    uint64_t pending = 0;  // ticket of the asynchronous batch still ingesting it, or 0
};

// Staging area of keyframe ingest (device copy of the caller-order arrays + pinned mirror).
struct IngestStage {
    DevBuf dev;
    PinBuf host;
    std::vector<std::pair<size_t, size_t>> host_ranges;
    std::vector<uint32_t> src;  // first staged keypoint of each keyframe
    void release() { dev.release(); host.release(); }
};

// Launch choices of a batch's fused form that the autotuner makes (results never depend on
// them): queries per lane of a search warp's group (1: 32-query groups, 2: 64), persistent
// search CTAs, the L2 prefetch of a pair's descriptors, which branch the scheduler serves
// first (0 search, 1 store), dense node blocks from this run length (0 = off; only when the
// caller asks for the tuner's choice, dense_min -1), the dense kernel's split divisor.
struct Knobs {
    // (the store branch first by default: ingest -> fusion -> its copy is the batch's usual
    // critical chain)
    int qpl = 2, persist = 0, prefetch = 0, bprio = 1, dense_min = 0, dsplit_div = 1;
};

// Device and staging buffers of one batch, plus what the host needs to read its results.
struct BatchBuf {
    DevBuf items, masks, mp_pos, mp_normal, mp_desc, mp_min, mp_max, mp_skip, padded,
        counts, item_cmp, offsets, ncmp, counters, dense, scratch, dres, acc, pconst, pwords, pepos, work, points,
        point_ok, pwin, pacc, pdone, ents, povf, mp_block;
    uint32_t n_units = 0;          // search launch entries (split pairs twice)
    uint32_t ent_cap = 0;          // entry form: capacity of ents (entries; 0 = form not prepared)
    PinBuf h_stage, h_out;
    IngestStage ingest;            // keyframes entering the store with this batch
    IngestArgs ingest_args{};
    int n_new = 0;
    bool nbr_new = false;          // a neighbour of some pair enters with this batch
    std::vector<WorkItem> h_items;
    std::vector<int> item_nq, item_nt;
    std::vector<int> step_pair_begin, step_fuse_item, slots;
    std::vector<int> new_index;    // slot -> position among the new keyframes, -1 (work list)
    std::vector<int> pair_fwd_item;  // [pairs + 1] first forward-fusion item of each pair
    uint32_t n_bwd_items = 0;        // fusion items into the new keyframes
    uint32_t search_pad = 0;         // padded output entries of the search items
    bool any_fwd = false;            // some step asks for forward fusion
    uint32_t n_items = 0, n_search_items = 0, total_pad = 0;
    uint32_t res_total = 0, t_total = 0, fsn = 16;
    int n_steps = 0, n_pairs = 0, smem_n = 32;
    int threads = 256, lanes = 1, ctas = 0;
    Knobs knobs;                   // the fused form's launch choices (tune_batch)
    bool tuned = false;            // knobs measured or cached by the tuner
    int user_dense_min = 0;        // the caller's dense_min (-1: the tuner's choice)
    uint32_t dsplit_base = 1;      // dense kernel CTAs per pair before the tuner's divisor
    tm_search_params sp{};
    tm_fuse_params fp{};
    BatchArgs args{};
    cudaGraphExec_t graph = nullptr;        // kernels only
    cudaGraphExec_t graph_timed = nullptr;  // the same with events at the stage boundaries
    cudaEvent_t ev[8] = {};                 // stage boundaries (timed graph)
    cudaEvent_t join = nullptr;          // end of the search branch
    cudaStream_t paux = nullptr;         // search branch (beside the ingest)
    cudaEvent_t pfork = nullptr;         // start of the search branch
    cudaEvent_t ingest_done = nullptr;   // if set: recorded after the batch's ingest (async batches)
    bool allow_pending = false;          // may use keyframes that batches in flight still ingest
                                         // (an asynchronous batch, ordered after them)
    // one-shot batches (early_fork): the search branch forks right after the work list and the
    // masks are uploaded, and the map points are copied on mcopy, which the fusion kernel
    // awaits (mready); forked / mp_async say that prepare_batch did so for the next enqueue
    bool early_fork = false, forked = false, mp_async = false;
    cudaStream_t mcopy = nullptr;
    cudaEvent_t mpre = nullptr, mready = nullptr;
    std::vector<void *> pointers() const;
    void release();
};

}  // namespace tmap

namespace tmap {
// Keyframe id -> store slot: open addressing with linear probing (the store's hottest host
// lookup: one per pair and step of every batch).  The subset of std::unordered_map's
// interface the library uses: find / end / count / erase / operator[] / size.
class IdMap {
  public:
    struct Entry {
        uint64_t first;
        int second;
        uint8_t state;  // 0 empty, 1 full, 2 erased
    };
    using iterator = Entry *;
    IdMap() { rehash(64); }
    iterator end() const { return nullptr; }
    size_t size() const { return n_; }
    iterator find(uint64_t k) const {
        size_t i = hash(k) & mask_;
        for (;;) {
            Entry &e = tab_[i];
            if (e.state == 0) return nullptr;
            if (e.state == 1 && e.first == k) return &e;
            i = (i + 1) & mask_;
        }
    }
    size_t count(uint64_t k) const { return find(k) ? 1 : 0; }
    int &operator[](uint64_t k) {
        if (Entry *e = find(k)) return e->second;
        if (2 * (used_ + 1) > tab_.size()) rehash(2 * n_ + 2 > tab_.size() / 2 ? 2 * tab_.size() : tab_.size());
        size_t i = hash(k) & mask_;
        while (tab_[i].state == 1) i = (i + 1) & mask_;
        if (tab_[i].state == 0) ++used_;
        tab_[i] = Entry{k, 0, 1};
        ++n_;
        return tab_[i].second;
    }
    void erase(iterator it) {
        if (!it || it->state != 1) return;
        it->state = 2;
        --n_;
    }
    size_t erase(uint64_t k) {
        iterator it = find(k);
        if (!it) return 0;
        erase(it);
        return 1;
    }

  private:
    static size_t hash(uint64_t k) {  // splitmix64 finaliser
        k ^= k >> 30;
        k *= 0xbf58476d1ce4e5b9ull;
        k ^= k >> 27;
        k *= 0x94d049bb133111ebull;
        k ^= k >> 31;
        return (size_t)k;
    }
    // table of `cap` entries (a power of two) holding the live entries; erased ones are dropped
    void rehash(size_t cap) {
        std::vector<Entry> old;
        old.swap(tab_);
        tab_.assign(cap, Entry{0, 0, 0});
        mask_ = cap - 1;
        n_ = used_ = 0;
        for (const Entry &e : old)
            if (e.state == 1) {
                size_t i = hash(e.first) & mask_;
                while (tab_[i].state != 0) i = (i + 1) & mask_;
                tab_[i] = e;
                ++n_;
                ++used_;
            }
    }
    mutable std::vector<Entry> tab_;  // (find hands out pointers to entries)
    size_t mask_ = 0, n_ = 0, used_ = 0;  // used_: full and erased entries (probe length)
};
}  // namespace tmap

struct tm_ctx {
    int device = 0;
    tm_camera cam{};
    int cap = 0;
    tmap::SlotLayout layout{};
    size_t slot_bytes = 0, budget = 0;
    int num_sms = 1;
    size_t max_smem = 0;  // opt-in shared memory per block
    tmap::CamConst camc{};
    std::mutex mu;
    tmap::IdMap ids;
    std::vector<tmap::Slot> slots;
    std::vector<int> free_slots;
    std::vector<void *> chunks;
    cudaStream_t stream = nullptr, capture_stream = nullptr;
    tmap::IngestStage ingest;
    tmap::BatchBuf batch;
    tmap::DevBuf mask_scratch;
    std::map<int, std::pair<int, int>> tuned;
    std::map<int, tmap::Knobs> tuned_knobs;
    tmap::Knobs last_knobs;
    int def_threads = 256, def_lanes = 1, last_threads = 256, last_lanes = 1, last_staged = -1;
    long long wait_limit = 4000000000ll;  // bound of device bulk-copy waits (SM cycles)
    uint32_t starve = 0;                  // test hook: bounded waits run out (no copy in flight)
    int force_threads = 0;                // test hook: threads per search CTA (0 = tuned)
    int force_prefetch = -1;              // test hook: search CTAs' L2 prefetch (-1 = tuned)
    int branch_prio = -1;                 // test hook: 0 search branch first, 1 store, 2 equal, -1 tuned
    int force_qpl = 0;                    // test hook: queries per lane of a search group (0 = tuned)
    long long entry_cap = 0;              // test hook: entry list capacity of the entry form (0 = sized
                                          // from the batch; TM_DEBUG_ENTRY_CAP)
    int force_persist = -1;               // test hook: persistent search CTAs (-1 = tuned)
    int split_min = 768;                  // pairs with at least this many queries take two search
                                          // CTAs in batches of fewer pairs than SMs; < 0: in any
                                          // batch (from -split_min); 0: none (TM_DEBUG_SPLIT_MIN)
    // host time of the phases of the last one-shot batch (tm_batch_last_host_times), in
    // microseconds: work list + uploads, launches, wait for the GPU and the result counts,
    // result downloads; t_counts marks the end of the third phase
    double host_us[4] = {0, 0, 0, 0};
    double t_counts = 0;
    // asynchronous one-shot batches (tm_batch_begin / tm_batch_finish): each on its own stream
    struct AsyncBatch {
        tmap::BatchBuf B;
        cudaStream_t s = nullptr;
        cudaEvent_t ingested = nullptr;   // after the batch's ingest (or its start)
        uint64_t ticket = 0;              // 0: free
        bool finishing = false;           // a tm_batch_finish is waiting for it (without the lock)
        std::vector<uint64_t> new_ids;    // the keyframes it stores (taken out again on failure)
    };
    AsyncBatch async[TM_BATCH_INFLIGHT];
    uint64_t async_next = 1;
    int async_last = -1;                  // the slot begun last
    ~tm_ctx();
};

namespace tmap {

tm_status fail(tm_status s, const char *fmt, ...);
tm_status cuda_fail(cudaError_t e, const char *what);
bool is_device_ptr(const void *p);
cudaStream_t pick_stream(tm_ctx *c, void *s);
tm_status validate_view(tm_ctx *c, const tm_keyframe_view &v);
// Where the five arrays of a packed keyframe set live, classified once for all its keyframes.
struct PackedSource {
    int kind = 0;                       // 1 device, 2 page-locked host, 3 pageable host
    const unsigned char *src[5] = {};   // desc, xy, angle, node, level (kind 2: device-mapped)
    size_t total = 0;                   // keypoints of all keyframes
};
// Checks a packed keyframe set of n keyframes (counts, null arrays, levels, one kind of memory
// per set) and gives its per-keyframe views (pointers into the packed arrays) and its source.
tm_status classify_packed(tm_ctx *c, const tm_keyframes_packed &p, int n, std::vector<tm_keyframe_view> &views,
                          PackedSource &src);
// Reserves n store slots (all or nothing) within the budget; caller holds c->mu.
tm_status alloc_slots_locked(tm_ctx *c, int n, std::vector<int> &got);
// Copies keyframes (host or device arrays) into staging buffers on stream s and fills the
// ingest kernel's arguments; enqueue_ingest also launches it.
tm_status stage_ingest(tm_ctx *c, IngestStage &st, int n, const tm_keyframe_view *kfs,
                       const int *slots, cudaStream_t s, IngestArgs &args, const PackedSource *pk = nullptr);
tm_status enqueue_ingest(tm_ctx *c, IngestStage &st, int n, const tm_keyframe_view *kfs,
                         const int *slots, cudaStream_t s);
tm_status store_add(tm_ctx *c, int n, const uint64_t *ids, const tm_keyframe_view *kfs,
                    cudaStream_t s, std::vector<int> &slots);
tm_status prepare_batch(tm_ctx *c, BatchBuf &B, const tm_step *steps, int n_steps,
                        const tm_batch_inputs *in, const tm_search_params &sp,
                        const tm_fuse_params &fp, cudaStream_t s);
tm_status enqueue_fused(tm_ctx *c, BatchBuf &B, int threads, int lanes, cudaStream_t s, bool timed = false);
tm_status enqueue_plain(tm_ctx *c, BatchBuf &B, int lanes, cudaStream_t s);
// t_counts: where to note when the counts arrived (default: c->t_counts, under c's lock)
tm_status fetch_results(tm_ctx *c, BatchBuf &B, tm_batch_result *r, cudaStream_t s, double *t_counts = nullptr);
tm_status tune_batch(tm_ctx *c, BatchBuf &B, const tm_step *steps, cudaStream_t s, bool measure);
void load_tuning(tm_ctx *c, const char *path);
// Threads per CTA used when no tuned value applies.
int default_threads(const tm_ctx *c, const BatchBuf &B);

}  // namespace tmap
