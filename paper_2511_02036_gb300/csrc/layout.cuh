// Device data layout of the keyframe store and of a batch (internal to the library).
//
// A keyframe occupies one fixed-size slot (Sec. IV-B: immutable keyframe data, resident
// until removal).  Inside a slot every array is SoA, 128-byte aligned, and the keypoints are
// stored grouped by BoW node: in ascending order of the node key (a bijective mix of the node
// id, stored in `node`), caller order within a node, so that a node's keypoints are a
// contiguous range read with consecutive 32-byte descriptor loads.  `bstart` indexes that
// order by the key's top kBucketBits bits (bucket b = positions bstart[b] .. bstart[b+1]), so
// a query finds its node's keypoints in one bucket.  `orig` maps a position back to the
// caller's keypoint index and `pos` is its inverse; `grid_start`/`grid_items` index positions
// by projection-grid cell.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace tmap {

constexpr int kLevels = 8;
constexpr int kBins = 30;
constexpr int kGridCols = 64;
constexpr int kGridRows = 48;
constexpr int kGridCells = kGridCols * kGridRows;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kBucketBits = 11;  // node-key buckets of a keyframe's node index
constexpr int kBuckets = 1 << kBucketBits;
constexpr int kFuseChunk = 512; // map points per fusion item (one CTA of the fusion kernel, two per thread)
constexpr int kQueryGroup = 64; // queries per search unit (one warp, two per lane)

__host__ __device__ constexpr size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// Slot header: 128 bytes.
struct KfHeader {
    int32_t n;
    int32_t cap;
    int32_t pad[2];
    double Tcw[12];
};

// Byte offsets of the arrays of a slot with capacity `cap` keypoints.
struct SlotLayout {
    size_t desc, xy, angle, node, orig, pos, level, grid_start, grid_items, bstart, bytes;
    __host__ __device__ static constexpr SlotLayout make(int cap) {
        SlotLayout L{};
        size_t o = align128(sizeof(KfHeader));
        L.desc = o;       o = align128(o + size_t(cap) * 32);
        L.xy = o;         o = align128(o + size_t(cap) * 8);
        L.angle = o;      o = align128(o + size_t(cap) * 4);
        L.node = o;       o = align128(o + size_t(cap) * 4);
        L.orig = o;       o = align128(o + size_t(cap) * 2);
        L.pos = o;        o = align128(o + size_t(cap) * 2);
        L.level = o;      o = align128(o + size_t(cap) * 1);
        L.grid_start = o; o = align128(o + size_t(kGridCells + 1) * 2);
        L.grid_items = o; o = align128(o + size_t(cap) * 2);
        L.bstart = o;     o = align128(o + size_t(kBuckets + 1) * 2);
        L.bytes = o;
        return L;
    }
};

// Typed view of one slot.
struct KfView {
    const KfHeader *hdr;
    const uint4 *desc;      // [n][2]
    const float2 *xy;
    const float *angle;
    const uint32_t *node;
    const uint16_t *orig;
    const uint16_t *pos;         // caller index -> position (inverse of orig)
    const uint8_t *level;
    const uint16_t *grid_start;  // [kGridCells + 1]
    const uint16_t *grid_items;  // sorted positions, grouped by cell
    const uint16_t *bstart;      // [kBuckets + 1] first position of each node-key bucket
    __host__ __device__ static KfView at(const unsigned char *base, const SlotLayout &L) {
        KfView v;
        v.hdr = reinterpret_cast<const KfHeader *>(base);
        v.desc = reinterpret_cast<const uint4 *>(base + L.desc);
        v.xy = reinterpret_cast<const float2 *>(base + L.xy);
        v.angle = reinterpret_cast<const float *>(base + L.angle);
        v.node = reinterpret_cast<const uint32_t *>(base + L.node);
        v.orig = reinterpret_cast<const uint16_t *>(base + L.orig);
        v.pos = reinterpret_cast<const uint16_t *>(base + L.pos);
        v.level = base + L.level;
        v.grid_start = reinterpret_cast<const uint16_t *>(base + L.grid_start);
        v.grid_items = reinterpret_cast<const uint16_t *>(base + L.grid_items);
        v.bstart = reinterpret_cast<const uint16_t *>(base + L.bstart);
        return v;
    }
};

// Raw (caller-order) keyframe arrays staged for ingest, concatenated over a batch.
struct IngestJob {
    unsigned char *slot;     // destination slot
    uint32_t src;            // first keypoint of this keyframe in the staged arrays
    int32_t n;
    double Tcw[12];
};

// A keyframe in page-locked host memory whose arrays a kernel copies into the staging area:
// desc, xy, angle, node, level (device addresses of the host pages), first staged keypoint, n.
struct GatherJob {
    const unsigned char *src[5];
    uint32_t dst;
    uint32_t n;
};

struct IngestArgs {
    const IngestJob *jobs;
    int32_t n_jobs;
    int32_t cap;
    const uint4 *desc;       // staged, caller order
    const float2 *xy;
    const float *angle;
    const uint32_t *node;
    const uint8_t *level;
    float cell_w_inv, cell_h_inv;  // grid cells per pixel
};

enum : uint32_t { kItemSearch = 0, kItemFuse = 1 };
// Device status word bits.
enum : uint32_t { kStatusTimeout = 1u };
constexpr uint32_t kItemTimeout = 0x80000000u;  // item_cmp flag: a bounded wait ran out

// An output item: a (new keyframe, neighbour) pair of a step, or up to kFuseChunk map points
// of a step fused into the step's new keyframe.  The query keyframe of a pair is read where it
// is: a stored keyframe from its slot (positions in node-key order, keys stored, `qorig` maps a
// position to the caller's index), a keyframe entering with the batch from its staged
// caller-order arrays (raw node ids, identity order), so that the search need not wait for its
// ingest.
struct WorkItem {
    const unsigned char *q;  // fuse: target keyframe slot
    const unsigned char *t;  // search: neighbour slot
    const uint4 *qdesc;      // search: Q's arrays in the order the search visits Q
    const float2 *qxy;
    const uint32_t *qnode;   //   node keys, or raw node ids if qraw
    const uint16_t *qorig;   //   caller index of each position, or null (identity)
    const float *qangle;
    uint32_t qraw;
    uint32_t kind;
    uint32_t out_off;        // first entry of this item's region in the padded output
    uint32_t a;              // search: byte offset of q mask (kNone: all free); fuse: first mp
    uint32_t b;              // search: byte offset of t mask;                   fuse: mp count
    uint32_t c;              // fuse: first mp of the step (output mp_idx = m - c);
                             // search: first entry of the pair's queries in BatchArgs::dres
    uint32_t nq, nt;         // search: keypoint counts
    uint32_t step;           // fuse: step index
    uint32_t cost;           // scheduling estimate
    uint32_t idx;            // search: logical index of the item (its counts / comparisons)
    uint32_t skip;           // fuse: byte offset in masks of the item's per-map-point skip
                             //   bytes (forward fusion), or kNone: the batch's mp_skip
    const double *pq, *pt;   // search: poses Tcw of Q and T (slot header, or the ingest job of a
                             // keyframe entering with the batch)
    float mdepth;            // search: T's median scene depth (0 = unknown; pair-baseline skip)
    uint32_t toff;           // search: the pair's first entry in the batch's per-target arrays
                             //   (BatchArgs::pepos; a multiple of 32, so toff / 32 indexes pwords)
};
static_assert(sizeof(WorkItem) == 128, "work records are 128 bytes");

// Per-pair constants written by the prep kernel: F (row-major, float32), the epipole in the
// neighbour (x, y; epipole rejection only), and 1.0 when the pair-baseline skip applies.
constexpr int kPairConst = 12;

constexpr size_t kBucketTableBytes = ((size_t(kBuckets + 1) * 2 + 15) / 16) * 16;

// Shared-memory carve of a search CTA (one pair) for a capacity of sn keypoints (a multiple
// of 32); the first five arrays arrive by bulk copies:
//   tkey   the neighbour's node keys
//   bst    its node-key bucket table
//   words  its eligibility bitmap (32 positions a word) with the eligible positions before
//          each word: uint2 (bits, count before), sn / 32 + 1 words (the last: 0, total)
//   epos   the eligible positions in node order
//   pc     the pair's constants (kPairConst floats)
//   win    per target: lowest (distance << 16 | caller query) among the accepted queries
//   qbits  kept matches, one bit per caller query; qpre: prefix counts of its words (+ total)
struct SearchStage {
    size_t tkey, bst, words, epos, pc, win, qbits, qpre, bytes;
    __host__ __device__ static constexpr SearchStage make(int sn) {
        SearchStage L{};
        size_t o = 0;
        L.tkey = o;  o = align128(o + size_t(sn) * 4);
        L.bst = o;   o = align128(o + kBucketTableBytes);
        L.words = o; o = align128(o + size_t(sn / 32 + 1) * 8);
        L.epos = o;  o = align128(o + size_t(sn) * 2);
        L.pc = o;    o = align128(o + size_t(kPairConst) * 4);
        L.win = o;   o = align128(o + size_t(sn) * 4);
        L.qbits = o; o = align128(o + size_t(sn / 32) * 4);
        L.qpre = o;  o = align128(o + size_t(sn / 32 + 1) * 4);
        L.bytes = o;
        return L;
    }
};

// Shared-memory carve of a fusion CTA: the target keyframe's grid and the keypoint arrays the
// window test reads, for a capacity of sn keypoints (a multiple of 16).
struct FuseStage {
    size_t xy, gstart, gitems, orig, level, bytes;
    static constexpr size_t kGridStartBytes = ((size_t(kGridCells + 1) * 2 + 15) / 16) * 16;
    __host__ __device__ static constexpr FuseStage make(int sn) {
        FuseStage L{};
        size_t o = 0;
        L.xy = o;     o = align128(o + size_t(sn) * 8);
        L.gstart = o; o = align128(o + kGridStartBytes);
        L.gitems = o; o = align128(o + size_t(sn) * 2);
        L.orig = o;   o = align128(o + size_t(sn) * 2);
        L.level = o;  o = align128(o + size_t(sn));
        L.bytes = o;
        return L;
    }
};

struct SearchConst {
    int32_t hamming_max, ratio_num, ratio_den;
    float epi_chi2;
    int32_t epipolar, resolve, rot_filter;
    int32_t dense_min;            // dense node blocks (tensor cores) from this run length; 0 = off
    float epipole_px;             // epipole rejection radius at level 0 (0 = off)
    int32_t rot_mode;             // 0: 30 bins of 12 degrees; 1: round(rot / 30)
    float baseline_min_ratio;     // pair skip: baseline / median depth below this (0 = off)
};

struct FuseConst {
    float chi2;
    int32_t hamming_max;
    float radius_scale;
};

struct CamConst {
    double fx, fy, cx, cy;
    double kinv[4];               // K^-1 entries 1/fx, -cx/fx, 1/fy, -cy/fy (float64 divisions)
    int32_t width, height;
    float cell_w_inv, cell_h_inv;
    static CamConst make(double fx, double fy, double cx, double cy, int32_t w, int32_t h) {
        CamConst c;
        c.fx = fx;
        c.fy = fy;
        c.cx = cx;
        c.cy = cy;
        c.kinv[0] = 1.0 / fx;
        c.kinv[1] = -cx / fx;
        c.kinv[2] = 1.0 / fy;
        c.kinv[3] = -cy / fy;
        c.width = w;
        c.height = h;
        c.cell_w_inv = (float)kGridCols / (float)w;
        c.cell_h_inv = (float)kGridRows / (float)h;
        return c;
    }
};

struct Out3 { int32_t a, b, c; };

// Arguments of the batch kernels (search, fuse, copy).
struct BatchArgs {
    const WorkItem *items;        // logical order (search items first, then fuse items)
    uint32_t n_items;
    uint32_t n_search;            // search items come first
    uint32_t n_bwd;               // then this many fusion items into the new keyframes; the
                                  // rest fuse the new keyframes' map points into neighbours
    const WorkItem *sitems;       // the search items in launch order (largest pairs first)
    uint32_t fsn;                 // fusion stage capacity (largest target, rounded to 16)
    uint32_t *counters;           // [2] status of the last run (kStatusTimeout)
    const uint8_t *masks;         // caller-order eligibility masks
    const float *mp_pos, *mp_normal, *mp_min, *mp_max;
    uint32_t n_mp;                // map points of the batch
    const uint4 *mp_desc;
    const uint8_t *mp_skip;
    Out3 *padded;                 // per-item regions
    uint32_t *counts;             // [n_items]
    uint32_t *item_cmp;           // [n_items] comparisons of the item | kItemTimeout
    uint32_t *offsets;            // [n_items + 1] exclusive scan of counts
    unsigned long long *ncmp;     // [3] search, fuse, forward-fuse comparisons (written by copy)
    Out3 *dense;                  // compacted output
    SearchConst sp;
    FuseConst fp;
    CamConst cam;
    int32_t cap;                  // slot capacity (keypoints)
    SlotLayout L;                 // array offsets of a slot of that capacity
    int32_t sn;                   // search stage capacity: largest keypoint count of the batch's
                                  // pairs, rounded to 32
    long long wait_limit;         // bound of a bulk-copy wait, SM clock cycles
    uint32_t starve;              // test hook: after the copies, await a barrier nothing arrives
                                  // at, so that the bounded wait runs out
    int32_t triangulate;          // 1: tri_kernel over the match lists
    double tri_cos_max, tri_chi2, tri_ratio;
    float *points;                // [matches][3] triangulated points (triangulate)
    uint8_t *point_ok;            // [matches] accepted as new map points
    uint2 *dres;                  // [sum of nq over search items] per-query (best key, second) of
                                  // dense queries, at WorkItem::c + position
    uint2 *acc;                   // [sum of nq over search items] accepted queries of each pair,
                                  // listed from WorkItem::c: (target position << 16 | caller,
                                  // bin << 25 | distance << 16 | target caller index)
    uint32_t l2_prefetch;         // search CTAs ask L2 to prefetch their pair's descriptors
    uint32_t qpl;                 // search: queries per lane of a warp's group (1 or 2)
    uint32_t persist;             // search: resident CTAs take pairs from *work (else CTA per pair)
    uint32_t *work;               // next pair of the persistent search (reset by the copy kernel)
    float *pconst;                // [n_search][kPairConst] per-pair constants (prep kernel)
    uint2 *pwords;                // per pair from toff / 32: eligibility words (bits, count before)
                                  //   and one closing word (0, eligible total)
    uint16_t *pepos;              // per pair from toff: the eligible positions in node order
    // split pairs (a pair's query groups over two search CTAs; WorkItem::step = part | parts << 8
    // for search items): the per-target winners of a split pair live in pwin from toff (the
    // prep kernel resets them), each part's accepted count in pacc[2 idx + part], and the last
    // part to finish (pdone[idx], counted by atomics) finalizes the pair
    uint32_t *pwin;
    uint32_t *pacc;
    uint32_t *pdone;
    uint32_t n_units;             // search launch entries (pairs, split pairs twice)
    uint32_t dsplit;              // dense kernel CTAs per search item
    // entry form (qpl 4): a join pass lists every (query, candidate) entry of the batch in ents
    // (launch entry, query position << 16 | target position), counted by *nents (reset by the
    // prep kernel); each entry is evaluated by its own thread, folding into its query's
    // (best key, second) in dres; a finalize pass reads those.  Entries past ent_cap are not
    // written and their pair is flagged in povf (its finalize searches it in rounds instead).
    uint2 *ents;
    uint32_t *nents;
    uint32_t ent_cap;
    uint32_t *povf;
};

}  // namespace tmap
