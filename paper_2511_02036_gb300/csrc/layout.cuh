// Device data layout of the keyframe store and of a batch (internal to the library).
//
// A keyframe occupies one fixed-size slot (Sec. IV-B: immutable keyframe data, resident
// until removal).  Inside a slot every array is SoA, 128-byte aligned, and the keypoints are
// stored in BoW-node order (stable: ties keep the caller's order), so that a node bucket is
// a contiguous range and the candidates of one query are read with consecutive 32-byte
// descriptor loads.  `orig` maps a sorted position back to the caller's keypoint index.
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
constexpr int kFuseChunk = 256;         // map points per fusion item, unstaged kernel
constexpr int kFuseChunkStaged = 2048;  // map points per fusion item, staged kernel

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
    size_t desc, xy, angle, node, orig, level, grid_start, grid_items, bytes;
    __host__ __device__ static constexpr SlotLayout make(int cap) {
        SlotLayout L{};
        size_t o = align128(sizeof(KfHeader));
        L.desc = o;       o = align128(o + size_t(cap) * 32);
        L.xy = o;         o = align128(o + size_t(cap) * 8);
        L.angle = o;      o = align128(o + size_t(cap) * 4);
        L.node = o;       o = align128(o + size_t(cap) * 4);
        L.orig = o;       o = align128(o + size_t(cap) * 2);
        L.level = o;      o = align128(o + size_t(cap) * 1);
        L.grid_start = o; o = align128(o + size_t(kGridCells + 1) * 2);
        L.grid_items = o; o = align128(o + size_t(cap) * 2);
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
    const uint8_t *level;
    const uint16_t *grid_start;  // [kGridCells + 1]
    const uint16_t *grid_items;  // sorted positions, grouped by cell
    __host__ __device__ static KfView at(const unsigned char *base, const SlotLayout &L) {
        KfView v;
        v.hdr = reinterpret_cast<const KfHeader *>(base);
        v.desc = reinterpret_cast<const uint4 *>(base + L.desc);
        v.xy = reinterpret_cast<const float2 *>(base + L.xy);
        v.angle = reinterpret_cast<const float *>(base + L.angle);
        v.node = reinterpret_cast<const uint32_t *>(base + L.node);
        v.orig = reinterpret_cast<const uint16_t *>(base + L.orig);
        v.level = base + L.level;
        v.grid_start = reinterpret_cast<const uint16_t *>(base + L.grid_start);
        v.grid_items = reinterpret_cast<const uint16_t *>(base + L.grid_items);
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

// Shared-memory carve of the staged batch kernel for a stride of sn keypoints (a multiple
// of 16).  A search item stages both keyframes of its pair; a fusion item stages its target
// keyframe and its projection grid.  The two carves overlay the same memory.
struct StageLayout {
    size_t tdesc, qdesc, txy, qxy, tnode, qnode, tangle, qangle, win, torig, qorig, tlevel,
        tmask, qmask, search_bytes;
    size_t fdesc, fxy, forig, flevel, fgstart, fgitems, fuse_bytes, bytes;
    static constexpr size_t kGridStartBytes = ((size_t(kGridCells + 1) * 2 + 15) / 16) * 16;
    __host__ __device__ static StageLayout make(int sn) {
        StageLayout L;
        const size_t n = (size_t)sn;
        size_t o = 0;
        L.tdesc = o;  o = align128(o + n * 32);
        L.qdesc = o;  o = align128(o + n * 32);
        L.txy = o;    o = align128(o + n * 8);
        L.qxy = o;    o = align128(o + n * 8);
        L.tnode = o;  o = align128(o + n * 4);
        L.qnode = o;  o = align128(o + n * 4);
        L.tangle = o; o = align128(o + n * 4);
        L.qangle = o; o = align128(o + n * 4);
        L.win = o;    o = align128(o + n * 4);
        L.torig = o;  o = align128(o + n * 2);
        L.qorig = o;  o = align128(o + n * 2);
        L.tlevel = o; o = align128(o + n);
        L.tmask = o;  o = align128(o + n);
        L.qmask = o;  o = align128(o + n);
        L.search_bytes = o;
        o = 0;
        L.fdesc = o;   o = align128(o + n * 32);
        L.fxy = o;     o = align128(o + n * 8);
        L.forig = o;   o = align128(o + n * 2);
        L.flevel = o;  o = align128(o + n);
        L.fgstart = o; o = align128(o + kGridStartBytes);
        L.fgitems = o; o = align128(o + n * 2);
        L.fuse_bytes = o;
        L.bytes = L.search_bytes > L.fuse_bytes ? L.search_bytes : L.fuse_bytes;
        return L;
    }
};

enum : uint32_t { kItemSearch = 0, kItemFuse = 1 };
// Device status word bits.
enum : uint32_t { kStatusTimeout = 1u };

// One unit of the persistent launch: a (new keyframe, neighbour) pair, or a chunk of up to
// kFuseChunk map points fused into a keyframe.
struct WorkItem {
    const unsigned char *q;  // search: new keyframe slot; fuse: target keyframe slot
    const unsigned char *t;  // search: neighbour slot; fuse: unused
    uint32_t kind;
    uint32_t out_off;        // first entry of this item's region in the padded output
    uint32_t a;              // search: byte offset of q mask (kNone: all free); fuse: first mp
    uint32_t b;              // search: byte offset of t mask;                   fuse: mp count
    uint32_t c;              // fuse: first mp of the step (output mp_idx = m - c)
    uint32_t cost;           // scheduling estimate
};

struct SearchConst {
    int32_t hamming_max, ratio_num, ratio_den;
    float epi_chi2;
    int32_t epipolar, resolve, rot_filter;
};

struct FuseConst {
    float chi2;
    int32_t hamming_max;
    float radius_scale;
};

struct CamConst {
    double fx, fy, cx, cy;
    int32_t width, height;
    float cell_w_inv, cell_h_inv;
};

struct Out3 { int32_t a, b, c; };

// Arguments of the persistent batch kernel and its copy pass.
struct BatchArgs {
    const WorkItem *items;        // logical order (search items first, then fuse items)
    const uint32_t *order;        // execution order (largest first)
    uint32_t n_items;
    uint32_t *counters;           // [0] next item, [1] CTAs done, [2] status
    const uint8_t *masks;
    const float *mp_pos, *mp_normal, *mp_min, *mp_max;
    const uint4 *mp_desc;
    const uint8_t *mp_skip;
    Out3 *padded;                 // per-item regions
    uint32_t *counts;             // [n_items]
    uint32_t *offsets;            // [n_items + 1] exclusive scan of counts, written by last CTA
    unsigned long long *ncmp;     // [2] search, fuse comparisons
    float *pair_F;                // [n_search][9] fundamental matrix of each search item
    uint32_t n_search;            // search items come first in logical order
    Out3 *dense;                  // compacted output
    uint32_t *status;             // device error word
    SearchConst sp;
    FuseConst fp;
    CamConst cam;
    int32_t cap;                  // slot capacity (keypoints)
    int32_t lanes;                // lanes per query
    int32_t staged;               // 1: TMA-staged kernel, sn = stage stride
    int32_t sn;
};

}  // namespace tmap
