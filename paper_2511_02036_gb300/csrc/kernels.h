// Host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "layout.cuh"

namespace tmap {

// Keyframe ingest: one CTA per keyframe sorts its keypoints by BoW node and builds the
// projection-grid index inside its slot.
size_t ingest_smem_bytes(int cap);
// prio: scheduling priority of the launch (0 = the stream's; lower numbers are higher
// priority, within cudaDeviceGetStreamPriorityRange).
cudaError_t launch_ingest(const IngestArgs &a, cudaStream_t s, int prio = 0);
// Copies keyframes from page-locked host memory into the staging area `base` (array offsets
// offs: desc, xy, angle, node, level), one CTA per job.
cudaError_t launch_stage_gather(const GatherJob *jobs, int n, unsigned char *base, const size_t offs[5],
                                cudaStream_t s);

// Batch pipeline: prep (CTA per pair: F, eligibility), search (CTA per pair), fuse (CTA per
// 256 map points), copy.
size_t search_smem_bytes(int sn);
int search_ctas_per_sm(const BatchArgs &a);
cudaError_t launch_prep(const BatchArgs &a, cudaStream_t s, int prio = 0);
// The form a search launch gets: a.qpl and a.persist reset to 2 and 0 for the gate
// configurations that only have that form.
void search_form(BatchArgs &a);
// ctas: CTAs of a persistent launch (a.persist; one per pair otherwise)
cudaError_t launch_search(const BatchArgs &a, int ctas, cudaStream_t s, int prio = 0);
// Dense node blocks on the tensor cores (a.sp.dense_min > 0): a.n_search * a.dsplit CTAs;
// writes a.dres, which launch_search then reads (same stream, before it).
size_t dense_smem_bytes();
cudaError_t launch_dense(const BatchArgs &a, cudaStream_t s, int prio = 0);
cudaError_t launch_fuse(const BatchArgs &a, cudaStream_t s, int prio = 0);
// Part 0: the search items' records from dense record 0; part 1: the fusion items' from out0.
cudaError_t launch_copy(const BatchArgs &a, int part, uint32_t out0, int ctas, cudaStream_t s);
// Bounds-checking build: the first failed index check's site (0: none), optionally reset;
// enabled = false and site = 0 in the normal build.
cudaError_t debug_bounds(bool reset, uint32_t *site, bool *enabled);
// Triangulation of every match of the batch (a.triangulate; after the copy kernel: reads the
// offsets and the dense matches).
cudaError_t launch_tri(const BatchArgs &a, cudaStream_t s);

// Integer-pipe rate probe: `ctas` CTAs of 256 threads, each thread `iters` rounds of 8
// operations (mode 0 popc, 1 lop3, 2 one register-resident 256-bit Hamming distance per round);
// sink: one word per thread.
cudaError_t launch_int_rate(int mode, int ctas, int iters, uint32_t *sink, cudaStream_t s);

// Plain per-pair form: every stage of one pair is its own launch, with global scratch.
struct PairScratch {
    uint32_t *win;      // [cap]   per target: lowest (dist, query) key
    uint32_t *accq;     // [cap]   per sorted query: accepted (target, dist)
    uint32_t *res;      // [cap]   per original query: kept (target, dist, bin)
    uint32_t *hist;     // [32]    rotation histogram
    uint32_t *running;  // [2]     running output offset, spare
};
size_t pair_scratch_bytes(int cap);
PairScratch pair_scratch_at(void *base, int cap);
// Runs one pair: dense output appended at *running; pair_offset[0] receives the start.
cudaError_t launch_pair_plain(const unsigned char *q, const unsigned char *t, const uint8_t *mq,
                              const uint8_t *mt, int nq, int nt, int cap, const SearchConst &sp,
                              const CamConst &cam, const PairScratch &scr, Out3 *dense,
                              uint32_t *pair_offset, unsigned long long *ncmp, int lanes,
                              cudaStream_t s, float t_median_depth = 0.0f);
// Plain fusion: one thread per map point, then an ordered compaction appended at *running;
// offset_out[0] receives the start.
cudaError_t launch_fuse_plain(const unsigned char *t, int cap, const float *pos,
                              const float *normal, const uint4 *desc, const float *mn,
                              const float *mx, const uint8_t *skip, int n, const FuseConst &fp,
                              const CamConst &cam, uint32_t *res, Out3 *dense, uint32_t *running,
                              uint32_t *offset_out, unsigned long long *ncmp, cudaStream_t s);

}  // namespace tmap
