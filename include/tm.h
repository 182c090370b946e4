/*
 * tm -- GB300-native keypoint correspondence search and map-point fusion search for the
 * local-mapping stage of visual SLAM (TurboMap, Hosseininejad et al., arXiv 2511.02036).
 *
 * C ABI.  Plain pointers and sizes only.  Every function returns a tm_status; on failure
 * tm_last_error() returns a thread-local message and no output is written, except where a
 * function says otherwise (TM_ERR_CAPACITY reports the required size).
 *
 * Pointers marked "host or device" may point to pageable or pinned host memory or to device
 * memory of the context's GPU (unified addressing decides).  `stream` is a cudaStream_t of the
 * context's device, or NULL for the context's own stream.  Unless stated otherwise a call is
 * synchronous: it returns after its results are in the caller's buffers, and inputs may be
 * reused as soon as it returns.
 *
 * Units of work (Sec. IV):
 *   keyframe store    Sec. IV-B: the immutable part of a keyframe (keypoints, descriptors,
 *                     BoW nodes, pose) is copied to the GPU once, when the keyframe enters
 *                     local mapping, and stays resident until it is removed.
 *   search            Sec. IV-C: correspondence search of a new keyframe against each of its
 *                     neighbours -- descriptor comparisons validated by the epipolar
 *                     constraint, all neighbours in parallel, triangulation left to the caller.
 *   fuse              Sec. IV-D: for each map point of a batch, the most similar keypoint of a
 *                     keyframe within the projection window; merging is left to the caller.
 *   batch / server    many local-mapping steps in one launch, and a continuous-batching loop.
 *
 * The matching rules (BoW buckets, Hamming <= 50, ratio 0.6, epipolar chi2 3.84 sigma^2,
 * one match per target keypoint, 30-bin rotation histogram keeping the top three bins,
 * window 3*scale with chi2 5.99 sigma^2) are not spelled out by the paper; they are the
 * readings stated in the repository's design notes and are parameters below.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tm_status;
#define TM_OK 0
#define TM_ERR_INVALID_ARG 1 /* bad pointer, size or parameter                              */
#define TM_ERR_NOT_FOUND 2   /* unknown keyframe id                                         */
#define TM_ERR_EXISTS 3      /* keyframe id already stored                                  */
#define TM_ERR_NO_MEMORY 4   /* store full (slots or memory budget) or device allocation    */
#define TM_ERR_CAPACITY 5    /* output buffer too small; required sizes are reported        */
#define TM_ERR_CUDA 6        /* CUDA runtime error (message in tm_last_error)               */
#define TM_ERR_TIMEOUT 7     /* a bounded wait ran out                                      */
#define TM_ERR_BUSY 8        /* keyframe referenced by a live plan; server queue full       */

#define TM_DESC_BYTES 32       /* 256-bit binary descriptor                                 */
#define TM_LEVELS 8            /* pyramid levels, scale factor 1.2                          */
#define TM_MAX_KP_LIMIT 8192   /* largest per-keyframe keypoint capacity                    */

typedef struct tm_ctx tm_ctx;
typedef struct tm_plan tm_plan;
typedef struct tm_server tm_server;

/* Largest image side accepted (pixels).  The fusion window's grid cells are found with a
 * fixed 0.01 px margin, which bounds the float32 rounding of the window test for images up to
 * this size. */
#define TM_MAX_IMAGE_SIZE 16384

/* Pinhole camera shared by all keyframes of a context. */
typedef struct {
    int32_t width, height; /* image size in pixels, 1 .. TM_MAX_IMAGE_SIZE                  */
    double fx, fy, cx, cy; /* intrinsics in pixels                                         */
} tm_camera;

/* One keyframe's immutable data (Sec. IV-B), n keypoints in the caller's order.  Keypoint
 * indices reported by every call refer to this order.  Arrays: host or device. */
typedef struct {
    int32_t n;              /* 0 .. max_kp of the context                                   */
    const uint8_t *desc;    /* [n][32] descriptor bytes                                     */
    const float *xy;        /* [n][2]  pixel coordinates                                    */
    const float *angle;     /* [n]     orientation, degrees in [0, 360)                     */
    const uint8_t *level;   /* [n]     pyramid level 0..7                                   */
    const uint32_t *node;   /* [n]     BoW vocabulary node id                               */
    double Tcw[12];         /* row-major 3x4 [R | t], world -> camera                       */
} tm_keyframe_view;

/* A batch of map points (Sec. IV-D: the map-point data a stage needs, gathered by the
 * caller and transferred in one step).  Arrays: host or device. */
typedef struct {
    int32_t n;
    const float *pos;       /* [n][3] world position                                        */
    const float *normal;    /* [n][3] unit mean viewing direction                           */
    const uint8_t *desc;    /* [n][32] representative descriptor                            */
    const float *min_dist;  /* [n] scale-invariance distance range                          */
    const float *max_dist;  /* [n]                                                          */
    const uint8_t *skip;    /* [n] or NULL: 1 = already observed by the target keyframe     */
} tm_mappoint_view;

#define TM_MODE_FUSED 0      /* all pairs and map points of the call in one launch sequence
                                (search kernel: a CTA per pair; fusion; copy; default)     */
#define TM_MODE_PER_PAIR 1   /* plain form: one pair at a time, one launch per stage        */

typedef struct {
    int32_t hamming_max;    /* accept best <= hamming_max (50)                              */
    int32_t ratio_num;      /* accept ratio_den*best < ratio_num*second (3, 5);             */
    int32_t ratio_den;      /*   ratio_num = 0 disables the ratio test                      */
    float epi_chi2;         /* epipolar gate: dist^2 < epi_chi2 * 1.2^(2*level_T) (3.84)    */
    int32_t epipolar;       /* 1 = apply the epipolar gate                                  */
    int32_t resolve;        /* 1 = one match per target keypoint                            */
    int32_t rot_filter;     /* 1 = 30-bin rotation-histogram filter                         */
    int32_t mode;           /* TM_MODE_FUSED or TM_MODE_PER_PAIR                            */
    int32_t lanes_per_query;/* TM_MODE_PER_PAIR: lanes per query 1, 2, 4, 8, 16 or 32 (0 = 1);
                               TM_MODE_FUSED spreads each 32-query group's candidates over
                               its warp's lanes and ignores it                              */
    int32_t dense_min;      /* TM_MODE_FUSED: a query whose BoW node holds >= dense_min
                               keypoints of the neighbour is compared with all of them on
                               the tensor cores (descriptors as +-1 fp8 vectors, Hamming =
                               (256 - dot) / 2, exact); same results.  0 = off (default),
                               -1 = the autotuner's choice (plans), else >= 16.  Worth it for dense nodes (~64 and more); each
                               call with it on runs one more kernel.  TM_MODE_PER_PAIR
                               ignores it.                                                   */
    /* ORB-family variants (0 = off, the defaults): */
    float epipole_px;       /* drop a candidate whose squared distance to the epipole (the
                               new keyframe's centre projected into the neighbour) is below
                               epipole_px^2 * 1.2^level_T (ORB-SLAM uses 10; monocular)      */
    int32_t rot_mode;       /* rotation bins: 0 = 30 bins of 12 degrees, floor(rot / 12);
                               1 = ORB-family round(rot * (1/30)), bins 0..12 used          */
    float baseline_min_ratio; /* skip a pair whose baseline (distance between the camera
                               centres) over the neighbour's median scene depth is below
                               this (tm_step.nbr_median_depth; ORB-SLAM: 0.01)             */
} tm_search_params;

typedef struct {
    float chi2;             /* reprojection gate e^2 <= chi2 * 1.2^(2*level) (5.99)         */
    int32_t hamming_max;    /* (50)                                                         */
    float radius_scale;     /* window half-width radius_scale * 1.2^predicted_level (3.0)   */
} tm_fuse_params;

/* A correspondence: keypoint q_idx of the new keyframe and t_idx of the neighbour. */
typedef struct { int32_t q_idx, t_idx, dist; } tm_match;
/* A fusion candidate: map point mp_idx (index within its batch) and keypoint kp_idx. */
typedef struct { int32_t mp_idx, kp_idx, dist; } tm_fuse_match;

typedef struct {
    int32_t device, max_kp, slots_used, slots_free_in_budget;
    size_t slot_bytes, bytes_reserved, budget_bytes;
} tm_store_stats;

/* Defaults: the readings of the design notes (50, 3/5, 3.84, all gates on, fused mode,
 * lanes 0; 5.99, 50, 3.0). */
void tm_search_params_default(tm_search_params *p);
void tm_fuse_params_default(tm_fuse_params *p);

/* ---------------------------------------------------------------------------- context
 * Creates a context on `device` (made current for the calling thread).  max_kp (1 ..
 * TM_MAX_KP_LIMIT) fixes the per-keyframe slot size.  mem_budget_bytes bounds the keyframe
 * store; 0 = admit by the free device memory at the time of each allocation, keeping 1 GiB
 * in reserve.  The context owns all device memory it allocates; destroy frees it. */
tm_status tm_ctx_create(int device, const tm_camera *cam, int32_t max_kp,
                        size_t mem_budget_bytes, tm_ctx **out);
tm_status tm_ctx_destroy(tm_ctx *ctx);
const char *tm_last_error(void);
tm_status tm_store_get_stats(tm_ctx *ctx, tm_store_stats *out);

/* ---------------------------------------------------------------------------- store (Sec. IV-B)
 * Copies the keyframe into a device slot, then builds on the GPU its node-sorted keypoint
 * order (BoW buckets) and its 64x48 projection-grid index.  TM_ERR_EXISTS if the id is
 * stored, TM_ERR_NO_MEMORY if no slot fits the budget (nothing is stored then). */
tm_status tm_store_add_keyframe(tm_ctx *ctx, uint64_t kf_id, const tm_keyframe_view *kf,
                                void *stream);
/* Makes sure at least n_slots keyframe slots are allocated and free (one allocation for the
 * missing ones, within the memory budget), so that later additions -- a server's admissions
 * among them -- allocate no device memory.  TM_ERR_NO_MEMORY if the budget or the free
 * memory cannot hold them (the slots that could be allocated stay reserved). */
tm_status tm_store_reserve(tm_ctx *ctx, int32_t n_slots);
/* The same for n keyframes in one transfer and one launch; all or nothing. */
tm_status tm_store_add_keyframes(tm_ctx *ctx, int32_t n, const uint64_t *kf_ids,
                                 const tm_keyframe_view *kfs, void *stream);
/* Frees the slot (Sec. IV-B: resident until removed).  TM_ERR_BUSY while a plan uses it. */
tm_status tm_store_remove_keyframe(tm_ctx *ctx, uint64_t kf_id);
/* The same for n keyframes; all or nothing (TM_ERR_NOT_FOUND, TM_ERR_BUSY, or
 * TM_ERR_INVALID_ARG for an id given twice, and nothing is removed). */
tm_status tm_store_remove_keyframes(tm_ctx *ctx, int32_t n, const uint64_t *kf_ids);
/* Number of keypoints of a stored keyframe, or TM_ERR_NOT_FOUND. */
tm_status tm_store_keyframe_size(tm_ctx *ctx, uint64_t kf_id, int32_t *n);

/* ---------------------------------------------------------------------------- keyframe culling (Sec. IV-F)
 * Host-side observation counters: per map point, the number of keyframe observations at each
 * pyramid level (the paper keeps culling on the CPU and replaces the walk over each map point's
 * observation list by this array).  A map point of a keyframe, observed at level L there, counts
 * as redundant when at least th_obs other keyframes observe it at a level <= L + 1; the
 * keyframe is redundant when more than ratio * n of its n map points are (ORB-SLAM: th_obs 3,
 * ratio 0.9).  Map point ids 0 .. max_mps-1; a keyframe observes a map point at most once, and
 * its own observations are among the counts. */
typedef struct tm_obs_counter tm_obs_counter;
tm_status tm_obs_create(int32_t max_mps, tm_obs_counter **out);
tm_status tm_obs_destroy(tm_obs_counter *c);
/* Adds n observations (map point mp[k] seen at keypoint level level[k]).  TM_ERR_CAPACITY if a
 * counter would pass 65535 (the entries before it are added). */
tm_status tm_obs_add(tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level);
/* Removes n observations; all or nothing (TM_ERR_NOT_FOUND when one has nothing to remove). */
tm_status tm_obs_remove(tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level);
/* The redundancy test of one keyframe from its observations (its map points and their levels). */
tm_status tm_obs_redundant(tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level,
                           int32_t th_obs, float ratio, int32_t *n_redundant, int32_t *is_redundant);

/* ---------------------------------------------------------------------------- fuse-apply (Sec. IV-D)
 * The sequential stage after the parallel fusion search.  The search lists candidate duplicate
 * pairs (a map point, a keypoint of a target keyframe) from one state of the map; this stage
 * merges them one at a time in the caller's order (ORB-SLAM's local mapping: the new keyframe's
 * points into each neighbour, neighbour by neighbour, then the neighbours' points into the new
 * keyframe), re-checking every candidate against the map as it stands at that moment.
 *
 * A host-side map: per keyframe a keypoint -> map point table and each keypoint's pyramid level;
 * per map point its observations (keyframe, keypoint), whether it is live, and the point that
 * replaced it; and the culling counters (per map point and level, as tm_obs_*), updated
 * whenever an observation is added, moved or erased.  Applying candidate (m, T, j):
 *   - skipped if m is no longer live (replaced by an earlier candidate) or T already observes m;
 *   - else, if keypoint j of T has no map point, T observes m at j;
 *   - else, with p the point at j: the one with more observations survives (a tie keeps m),
 *     and the other is replaced: each of its observations (K, i) moves to the survivor, unless
 *     K already observes the survivor, in which case keypoint i of K loses its map point; the
 *     replaced point is no longer live and records the survivor.
 * Map point ids 0 .. max_mps-1 (a point exists from its first observation); keyframe ids are the
 * caller's (the store's, for one).  Every call validates all its arguments before it changes
 * anything: on an error the map is unchanged.  Calls on one map are serialised by a lock. */
typedef struct tm_map tm_map;
typedef struct {
    int32_t added;                /* keypoint had no map point: observation added             */
    int32_t merged_into_existing; /* the keypoint's point had more observations: m replaced   */
    int32_t replaced_existing;    /* m had as many or more: the keypoint's point replaced     */
    int32_t skipped_dead;         /* m was replaced by an earlier candidate                   */
    int32_t skipped_observed;     /* the target already observes m                           */
} tm_fuse_apply_stats;
tm_status tm_map_create(int32_t max_mps, tm_map **out);
tm_status tm_map_destroy(tm_map *m);
/* A keyframe of n_kp keypoints, level[n_kp] (0 .. TM_LEVELS-1; NULL: all 0), none with a map
 * point.  TM_ERR_EXISTS if the id is in the map. */
tm_status tm_map_add_keyframe(tm_map *m, uint64_t kf_id, int32_t n_kp, const uint8_t *level);
/* Erases the keyframe and all its observations (keyframe culling).  Points left without an
 * observation stay live.  TM_ERR_NOT_FOUND. */
tm_status tm_map_remove_keyframe(tm_map *m, uint64_t kf_id);
/* Keyframe kf_id observes map point mp[k] at keypoint kp[k] (points created by triangulation,
 * or seen by tracking).  TM_ERR_INVALID_ARG if a keypoint is out of range or already has a map
 * point, the keyframe already observes the point, a point is given twice, or it was replaced. */
tm_status tm_map_add_observations(tm_map *m, uint64_t kf_id, int32_t n, const int32_t *kp,
                                  const int32_t *mp);
/* Applies n candidates of one target keyframe kf_id in order: cand[k].kp_idx is a keypoint of
 * the target, and the map point is mp_ids[cand[k].mp_idx] (mp_ids[n_ids]: the batch's map point
 * ids, as tm_fuse and tm_batch_run index them) or, with mp_ids NULL, cand[k].mp_idx itself.
 * dist is not read.  TM_ERR_INVALID_ARG if an index is out of range or a point never existed.
 * stats (may be NULL) receives this call's counts. */
tm_status tm_map_fuse_apply(tm_map *m, uint64_t kf_id, int32_t n, const tm_fuse_match *cand,
                            const int32_t *mp_ids, int32_t n_ids, tm_fuse_apply_stats *stats);
/* out[n_kp]: the map point of each keypoint of the keyframe, -1 for none.  n_kp must equal the
 * keyframe's keypoint count. */
tm_status tm_map_keyframe_points(tm_map *m, uint64_t kf_id, int32_t n_kp, int32_t *out);
/* Per map point mp[k]: live[k] (1 live, 0 replaced, -1 never existed), current[k] (the live
 * point it now stands for, following replacements; -1 if it never existed) and n_obs[k] (its
 * number of observations; 0 once replaced).  Any output may be NULL. */
tm_status tm_map_point_info(tm_map *m, int32_t n, const int32_t *mp, int32_t *live,
                            int32_t *current, int32_t *n_obs);
/* Keyframe culling's redundancy test (as tm_obs_redundant) of keyframe kf_id over its map
 * points, read from the map's own counters. */
tm_status tm_map_redundant(tm_map *m, uint64_t kf_id, int32_t th_obs, float ratio,
                           int32_t *n_redundant, int32_t *is_redundant);

/* ---------------------------------------------------------------------------- search (Sec. IV-C)
 * Correspondence search of stored keyframe `kf` against stored neighbours nbrs[0..n_nbrs).
 *   q_free    [n_Q] or NULL   1 = the keypoint has no map point yet (eligible)     host/device
 *   nbr_free  [sum n_T] or NULL  the neighbours' masks concatenated in nbrs order  host/device
 *   out       host buffer of cap matches; pair k occupies out[pair_offsets[k] ..
 *             pair_offsets[k+1]), sorted by q_idx
 *   pair_offsets  host [n_nbrs + 1]
 *   n_comparisons host, optional: descriptor comparisons performed (same-node free pairs)
 * On TM_ERR_CAPACITY *n_out holds the number of matches and nothing else is written. */
tm_status tm_search_triangulation(tm_ctx *ctx, uint64_t kf, const uint64_t *nbrs,
                                  int32_t n_nbrs, const tm_search_params *params,
                                  const uint8_t *q_free, const uint8_t *nbr_free,
                                  tm_match *out, size_t cap, size_t *n_out,
                                  int32_t *pair_offsets, uint64_t *n_comparisons,
                                  void *stream);

/* ---------------------------------------------------------------------------- fuse (Sec. IV-D)
 * Fusion search of the map points `mps` into stored keyframe `kf`: at most one candidate per
 * map point, sorted by mp_idx.  Several map points may name the same keypoint; the caller's
 * sequential merge decides.  n_comparisons counts (map point, keypoint) pairs inside the
 * window at an admissible level. */
tm_status tm_fuse(tm_ctx *ctx, uint64_t kf, const tm_mappoint_view *mps,
                  const tm_fuse_params *params, tm_fuse_match *out, size_t cap,
                  size_t *n_out, uint64_t *n_comparisons, void *stream);

/* ---------------------------------------------------------------------------- batches
 * Many local-mapping steps in one launch sequence.  Masks and map points of all steps are
 * passed once, concatenated (one transfer each); a step names its ranges in them. */
typedef struct {
    uint64_t kf_id;          /* new keyframe (stored)                                       */
    const uint64_t *nbr_ids; /* host [n_nbrs] stored neighbours                             */
    int32_t n_nbrs;
    int64_t q_free_off;      /* byte offset of the new keyframe's mask in masks, -1 = free  */
    int64_t nbr_free_off;    /* byte offset of the neighbours' concatenated masks, -1 = free*/
    int32_t mp_begin;        /* this step's map points are mps[mp_begin, mp_begin+mp_count) */
    int32_t mp_count;        /*   fused into kf_id; 0 = no fusion                           */
    /* Forward fusion (Sec. IV-D, the other direction): the new keyframe's own map points
     * mps[fwd_mp_begin, fwd_mp_begin+fwd_mp_count) fused into every neighbour.  fwd_skip_off:
     * byte offset in masks of n_nbrs x fwd_mp_count bytes, neighbour-major (1 = the map point
     * is already observed by that neighbour: skipped), or -1 = none skipped.  Read only when
     * fwd_mp_count > 0. */
    int32_t fwd_mp_begin;
    int32_t fwd_mp_count;
    int64_t fwd_skip_off;
    /* host [n_nbrs] or NULL: each neighbour's median scene depth, for the pair-baseline skip
     * (a depth <= 0 never skips) */
    const float *nbr_median_depth;
} tm_step;

/* Triangulation of the search's matches and their acceptance as new map points (Sec. III,
 * Map Point Creation: sufficient parallax, positive depth, low reprojection error, scale
 * consistency), run on the GPU over the batch's match lists.  Float32: normalized
 * coordinates (u - cx) / fx; world rays R^T (xn, yn, 1), kept iff 0 < cos(parallax) <
 * cos_parallax_max; the point is the midpoint of the rays' common perpendicular; depth > 0
 * and reprojection error^2 <= chi2 * 1.44^level in each view; distance ratio to the two
 * camera centres consistent with the scale ratio within ratio_factor. */
typedef struct {
    double cos_parallax_max;  /* (0.9998)                                                   */
    double chi2;              /* (5.991)                                                    */
    double ratio_factor;      /* (1.8 = 1.5 * 1.2)                                          */
} tm_triangulation_params;
void tm_triangulation_params_default(tm_triangulation_params *p);

/* Keyframes packed one after another, one array per field: keyframe i's keypoints are rows
 * n[0] + ... + n[i-1] onward of every array.  The same data as an array of tm_keyframe_view
 * (Sec. IV-B), in a form whose arrays are classified (host, page-locked host, device) and
 * moved once for all keyframes rather than once per keyframe.  Arrays: host or device, each
 * array wholly in one kind of memory. */
typedef struct {
    const int32_t *n;       /* host [count] keypoints per keyframe                           */
    const uint8_t *desc;    /* [sum n][32]                                                    */
    const float *xy;        /* [sum n][2]                                                     */
    const float *angle;     /* [sum n]                                                        */
    const uint8_t *level;   /* [sum n]                                                        */
    const uint32_t *node;   /* [sum n]                                                        */
    const double *Tcw;      /* host [count][12], row-major 3x4 per keyframe                   */
} tm_keyframes_packed;

typedef struct {
    const uint8_t *masks;    /* host or device, mask_bytes bytes (may be NULL if unused)    */
    size_t mask_bytes;
    tm_mappoint_view mps;    /* all steps' map points (n may be 0)                          */
    /* Keyframes entering the store with this batch (Sec. IV-B), e.g. the steps' new
     * keyframes: they are stored before the search runs, in the same launch sequence, and
     * stay stored afterwards.  Ids must not be stored yet.  A plan stages them once and
     * re-runs their ingest (same data, same slots) at every tm_plan_run, so that a run covers
     * keyframe entry + search + fusion.  Arrays: host or device. */
    int32_t n_new;
    const uint64_t *new_ids;          /* host [n_new]                                       */
    const tm_keyframe_view *new_kfs;  /* host [n_new], or NULL with new_packed below          */
    /* NULL, or triangulate every match of the batch (results in tm_batch_result.points). */
    const tm_triangulation_params *tri;
    /* The new keyframes packed (count = n_new), in place of new_kfs (which is then NULL);
     * NULL when new_kfs is used. */
    const tm_keyframes_packed *new_packed;
    /* NULL, or one allocation (page-locked host or device memory) that holds every array of
     * mps: the batch then uploads the block [mps_block, mps_block + mps_block_bytes) with one
     * copy (a transfer costs a few microseconds besides its bytes) and reads the arrays at
     * their offsets in it.  The offsets of pos, normal, min_dist and max_dist must be
     * multiples of 4 bytes and that of desc a multiple of 16; an array outside the block or
     * an offset off alignment is TM_ERR_INVALID_ARG.  The block must stay valid and unchanged
     * like the arrays themselves. */
    const void *mps_block;
    uint64_t mps_block_bytes;
} tm_batch_inputs;

/* Results, host buffers.  Search matches of all steps, step-major then neighbour order:
 * pair p (counting pairs over all steps) is matches[pair_offsets[p] .. pair_offsets[p+1]).
 * Fusion candidates of step s are fuse[fuse_offsets[s] .. fuse_offsets[s+1]), mp_idx
 * relative to the step's mp_begin.  Forward-fusion candidates of pair p (the step's new
 * keyframe's map points in neighbour p's keypoints) are fwd[fwd_offsets[p] ..
 * fwd_offsets[p+1]), mp_idx relative to the step's fwd_mp_begin; fwd and fwd_offsets may be
 * NULL when no step asks for forward fusion. */
typedef struct {
    tm_match *matches; size_t match_cap; size_t n_matches;
    int32_t *pair_offsets;   /* [total pairs + 1]                                           */
    tm_fuse_match *fuse; size_t fuse_cap; size_t n_fuse;
    int32_t *fuse_offsets;   /* [n_steps + 1]                                               */
    uint64_t n_comparisons_search, n_comparisons_fuse;
    tm_fuse_match *fwd; size_t fwd_cap; size_t n_fwd;
    int32_t *fwd_offsets;    /* [total pairs + 1]                                           */
    uint64_t n_comparisons_fwd;
    /* With triangulation: per match (same order as matches) its point, float32 x, y, z in
     * the world frame (0 when not accepted), and 1 when accepted as a new map point; both
     * match_cap entries, required then. */
    float *points;
    uint8_t *point_ok;
} tm_batch_result;

/* One-shot: upload, one launch sequence, download.  TM_ERR_CAPACITY sets n_matches and
 * n_fuse to the required sizes and writes nothing else.  On any failure the batch's new
 * keyframes are not stored. */
tm_status tm_batch_run(tm_ctx *ctx, const tm_step *steps, int32_t n_steps,
                       const tm_batch_inputs *in, const tm_search_params *sp,
                       const tm_fuse_params *fp, tm_batch_result *res, void *stream);
/* Asynchronous form of tm_batch_run, for producers that prepare the next batch while the
 * previous one transfers and runs.  tm_batch_begin checks and enqueues the batch (work list,
 * uploads, ingest of its new keyframes, launches) on a stream of its own and returns a ticket
 * without waiting; tm_batch_finish waits for that batch and copies its results, with
 * tm_batch_run's result rules.  At most TM_BATCH_INFLIGHT batches of a context are in flight
 * (TM_ERR_BUSY beyond); each slot keeps its device buffers once used.  A batch's GPU work starts after the ingest of the batch begun before
 * it, so a neighbour may be a keyframe that an earlier in-flight batch stores; their copies
 * and kernels otherwise overlap.  The caller's input arrays (host or device) must stay valid
 * and unchanged until tm_batch_finish returns; keyframes used by an in-flight batch cannot be
 * removed (TM_ERR_BUSY), and the keyframes it stores may be read only by later batches begun
 * with tm_batch_begin until it is finished (other calls that name them: TM_ERR_BUSY).  If tm_batch_finish reports an error, the batch's new keyframes are
 * taken out of the store again, except those that a batch still in flight reads.  Tickets are
 * finished in any order; an unknown ticket (or one that another thread is finishing) is
 * TM_ERR_NOT_FOUND.  tm_batch_finish waits for its batch and downloads the results without
 * holding the context, so one thread may begin batches (or call anything else on the context)
 * while another finishes earlier ones; the result buffers of concurrent finishes must differ. */
#define TM_BATCH_INFLIGHT 4
tm_status tm_batch_begin(tm_ctx *ctx, const tm_step *steps, int32_t n_steps,
                         const tm_batch_inputs *in, const tm_search_params *sp,
                         const tm_fuse_params *fp, uint64_t *ticket);
tm_status tm_batch_finish(tm_ctx *ctx, uint64_t ticket, tm_batch_result *res);
/* Host wall time of the phases of the context's last tm_batch_run, in microseconds: us[0]
 * the work list and the uploads (prepare), us[1] the launches, us[2] waiting for the GPU and
 * the result counts, us[3] the result downloads; after a tm_batch_finish, its own wait (us[2])
 * and downloads (us[3]) with us[0] = us[1] = 0.  Zeros before the first call. */
tm_status tm_batch_last_host_times(tm_ctx *ctx, double us[4]);

/* Prepared batch: uploads the inputs once and captures the launch in a CUDA graph; each
 * tm_plan_run replays it (asynchronous on `stream`, results stay on the device until
 * tm_plan_results).  The plan keeps its keyframes from being removed until destroyed. */
tm_status tm_plan_create(tm_ctx *ctx, const tm_step *steps, int32_t n_steps,
                         const tm_batch_inputs *in, const tm_search_params *sp,
                         const tm_fuse_params *fp, tm_plan **out);
tm_status tm_plan_run(tm_plan *plan, void *stream);
/* The same run from a second graph that also records CUDA events at the stage boundaries
 * (each event node adds a few microseconds), for tm_plan_stage_times. */
tm_status tm_plan_run_timed(tm_plan *plan, void *stream);
tm_status tm_plan_results(tm_plan *plan, tm_batch_result *res, void *stream);
/* Launch configuration the plan uses: threads per search CTA (autotuned), lanes per query (the
 * parameter as given), search CTAs (one per pair), kernels per run. */
tm_status tm_plan_info(tm_plan *plan, int32_t *threads, int32_t *lanes, int32_t *ctas,
                       int32_t *kernels_per_run);
/* Launch choices of a plan's fused form, made by the autotuner when the plan was created
 * (measured once per batch regime and cached per context, and in the file named by the
 * TM_TUNE_CACHE environment variable when set; a file whose first line names another key
 * layout is ignored) or fixed by tm_debug_set.  The regime: comparisons per query, fewer pairs
 * than SMs, dense blocks off / on / left to the tuner, epipole rejection.  Results never depend
 * on them.  For a plain per-pair plan every field is 0. */
typedef struct {
    int32_t queries_per_warp; /* queries a search warp takes at a time: 32 or 64                 */
    int32_t persistent;       /* 1: resident search CTAs take pairs from a work counter          */
    int32_t l2_prefetch;      /* 1: search CTAs prefetch their pair's descriptors into L2        */
    int32_t branch_priority;  /* CTAs placed first when SMs free up: 0 search, 1 store branch    */
    int32_t dense_min;        /* dense node blocks on the tensor cores from this run length; 0 off */
    int32_t dense_split;      /* dense kernel CTAs per pair (0 when off)                         */
    int32_t search_ctas;      /* CTAs of the search launch                                       */
    int32_t tuned;            /* 1: chosen by the tuner (measured or cached); 0: defaults        */
    int32_t per_lane;         /* 1: each lane walks its own queries' candidates (per-lane form);
                                 0: a warp's candidates spread over its lanes in rounds          */
    int32_t search_units;     /* search launch entries: pairs, a split pair counted twice        */
    int32_t entry_form;       /* 1: the entry form -- a join pass lists every (query, candidate)
                                 entry of the batch, one thread evaluates each, a finalize pass
                                 per pair reads the queries' states (three launches)            */
} tm_plan_tuning;
tm_status tm_plan_get_tuning(tm_plan *plan, tm_plan_tuning *out);

/* Device time of the stages of the plan's last run when it was a tm_plan_run_timed, from the
 * CUDA events recorded inside its graph (all zero otherwise).  The search branch (prep kernel:
 * per-pair F and eligibility; search kernel: one CTA per pair, all of Sec. IV-C) runs beside
 * the store branch (ingest -> fusion): ms[0] search kernel (between events recorded right
 * before and after it on its stream), ms[1] ingest, ms[2] fusion kernel, ms[3] from the later of
 * the search and fusion kernels' ends to the end of the run: each branch's offsets + copy of its
 * own records (and the triangulation kernel after the search's, when the batch triangulates), ms[4] the
 * dense-block kernel that precedes the search kernel (dense_min > 0; else 0), ms[5] the prep
 * kernel.  Waits for the run to finish. */
#define TM_PLAN_STAGES 6
tm_status tm_plan_stage_times(tm_plan *plan, float ms[TM_PLAN_STAGES]);
tm_status tm_plan_destroy(tm_plan *plan);

/* ---------------------------------------------------------------------------- test hooks
 * Settings of a context that later batches (tm_batch_run, new plans, the server) take, for
 * testing failure detection without faulting the GPU.  The search and fusion kernels wait for
 * their bulk copies into shared memory with a bounded wait; when it runs out, the kernel
 * records it, returns without touching the copied data, and the call reports TM_ERR_TIMEOUT.
 *   TM_DEBUG_WAIT_LIMIT    the bound in SM clock cycles (default 4e9, about 2 s)
 *   TM_DEBUG_STARVE_WAITS  non-zero: after its copies have landed, every such kernel also
 *                          awaits a barrier that nothing arrives at, so that the bound runs
 *                          out with no copy in flight; 0 restores normal operation
 * Launch choices that the autotuner otherwise makes, fixed so that tests can check every
 * choice against the oracle (results never depend on them):
 *   TM_DEBUG_SEARCH_THREADS threads per search CTA: 256; 0 = tuned (default)
 *   TM_DEBUG_L2_PREFETCH    1: search CTAs ask L2 to prefetch their pair's descriptors and
 *                           positions at start; 0 or -1 (default): they do not
 *   TM_DEBUG_BRANCH_PRIORITY which branch of a batch the scheduler serves first: 0 the search
 *                           branch, 1 the store branch (ingest, fusion), 2 neither; -1 = tuned
 *                           (default)
 *   TM_DEBUG_QUERIES_PER_LANE search warps take 32 (1) or 64 (2) queries at a time with their
 *                           candidates spread over the lanes in rounds, or 64 with each lane
 *                           walking its own two queries' candidates (3); or the entry form (4:
 *                           join, one thread per candidate entry, finalize; batches with the
 *                           default gates only); 0 = tuned (default)
 *   TM_DEBUG_ENTRY_CAP      entries the entry form's list holds (0 = four per query visit, at
 *                           least 2^20, grown by the tuner to a batch's count; at most 2^26);
 *                           a pair with entries past it is searched in rounds by its finalize
 *   TM_DEBUG_PERSISTENT     1: resident search CTAs take pairs from a work counter; 0: one CTA
 *                           per pair; -1 = tuned (default)
 *   TM_DEBUG_SPLIT_MIN      in batches of fewer pairs than SMs, pairs with at least this many
 *                           query keypoints are searched by two CTAs, each half of the queries,
 *                           the last to finish finalizing the pair (default 768; 0 = never; a
 *                           negative value -n splits pairs of n or more in any batch); fused
 *                           batches with the default gates only (no epipole rejection, no
 *                           dense blocks), and not with the persistent search
 * Errors: TM_ERR_INVALID_ARG (null context, unknown setting, value out of range). */
#define TM_DEBUG_WAIT_LIMIT 1
#define TM_DEBUG_STARVE_WAITS 2
#define TM_DEBUG_SEARCH_THREADS 3
#define TM_DEBUG_L2_PREFETCH 4
#define TM_DEBUG_BRANCH_PRIORITY 5
#define TM_DEBUG_QUERIES_PER_LANE 6
#define TM_DEBUG_PERSISTENT 7
#define TM_DEBUG_SPLIT_MIN 8
#define TM_DEBUG_ENTRY_CAP 9
tm_status tm_debug_set(tm_ctx *ctx, int32_t what, int64_t value);
/* Bounds-checking builds (compiled with -DTM_DEBUG_BOUNDS; the normal build sets *enabled = 0
 * and *site = 0): every index the kernels take from data (bucket tables, grid lists, match and
 * query lists) is checked against its array; *site is the first failed check (0 = none), and
 * the failed index was clamped into range.  reset = 1 clears it after reading.  Reads the
 * current device's status. */
tm_status tm_debug_bounds(int32_t reset, uint32_t *site, int32_t *enabled);

/* Measured peak rates of the integer operations a descriptor comparison is made of (the ALU
 * term of the roofline; Sec. IV-C's comparisons are XOR + population count over 256 bits):
 * a probe kernel on `device` keeps every SM busy with independent register chains and is
 * timed with CUDA events (best of three launches).
 *   popc_per_s     population counts per second (popc.b32)
 *   lop3_per_s     three-input logic operations per second (lop3.b32)
 *   hamming_per_s  register-resident 256-bit Hamming distances per second (8 xor, 8 popc
 *                  and their sum each)
 * Any output may be NULL.  Synchronous; allocates and frees 1.3 MB of device memory.
 * Errors: TM_ERR_INVALID_ARG (bad device), TM_ERR_CUDA. */
tm_status tm_measure_int_rates(int32_t device, double *popc_per_s, double *lop3_per_s, double *hamming_per_s);

/* ---------------------------------------------------------------------------- serving
 * Continuous batching.  A host thread admits submitted requests in arrival order as
 * in-flight batch slots and store memory allow, ingests their keyframes, and launches
 * each batch's search + fuse while earlier batches are still on the GPU (a ring of
 * streams).  A request's neighbours must be stored or belong to earlier requests.  A request
 * may also carry its new keyframe's own map points for forward fusion into each neighbour
 * (Sec. IV-D), and the server may triangulate every match (Sec. III), as tm_batch_run does. */
typedef struct {
    int32_t max_batch_requests;   /* requests per launch (64)                               */
    int32_t max_inflight_batches; /* batches on the GPU at once (3)                         */
    int32_t queue_capacity;       /* pending requests before submit returns TM_ERR_BUSY     */
    int32_t evict_after;          /* keep only the newest N keyframes of the stream, 0 = no */
    tm_search_params search;
    tm_fuse_params fuse;
    int32_t triangulate;          /* 1: triangulate and check every match (tri below)       */
    tm_triangulation_params tri;
} tm_server_config;

typedef struct {
    uint64_t kf_id;
    tm_keyframe_view kf;          /* copied at submit                                       */
    const uint64_t *nbr_ids;      /* copied at submit                                       */
    int32_t n_nbrs;
    const uint8_t *q_free;        /* [n] or NULL, copied                                    */
    const uint8_t *nbr_free;      /* [sum n_T] or NULL, copied                              */
    tm_mappoint_view mps;         /* fused into kf_id; copied (host arrays)                 */
    tm_mappoint_view fwd_mps;     /* kf_id's own map points, fused into every neighbour;
                                     copied; n = 0 for none (its skip array is not read)     */
    const uint8_t *fwd_skip;      /* [n_nbrs][fwd_mps.n] or NULL: 1 = that neighbour already
                                     observes the point (not fused into it); copied          */
    size_t nbr_free_bytes;        /* length of nbr_free (the neighbours' keypoints), or 0: the
                                     server looks the neighbours' sizes up (under the context's
                                     lock, which a batch being launched holds)                */
} tm_request;

typedef struct {
    int32_t done;                 /* 1 when complete                                        */
    tm_status status;
    int32_t n_matches, n_fuse;
    double t_submit, t_admit, t_done; /* seconds, monotonic clock                           */
    int32_t n_fwd;                /* forward-fusion candidates                              */
} tm_request_info;

void tm_server_config_default(tm_server_config *c);
tm_status tm_server_start(tm_ctx *ctx, const tm_server_config *cfg, tm_server **out);
/* Host arrays only.  *ticket identifies the request. */
tm_status tm_server_submit(tm_server *srv, const tm_request *req, uint64_t *ticket);
/* Non-blocking status; timeout_s > 0 waits at most that long for completion. */
tm_status tm_server_poll(tm_server *srv, uint64_t ticket, double timeout_s,
                         tm_request_info *info);
/* Copies a finished request's results (host buffers): matches [n_matches], pair_offsets
 * [n_nbrs+1], fuse [n_fuse], then forgets the ticket. */
tm_status tm_server_take(tm_server *srv, uint64_t ticket, tm_match *matches,
                         int32_t *pair_offsets, tm_fuse_match *fuse);
/* The same with the forward-fusion and triangulation results: fwd [n_fwd] with fwd_offsets
 * [n_nbrs + 1] (per neighbour, as pair_offsets), points [n_matches][3] float and point_ok
 * [n_matches] (only with triangulate in the configuration; else not written).  Any output may
 * be NULL. */
tm_status tm_server_take_ex(tm_server *srv, uint64_t ticket, tm_match *matches,
                            int32_t *pair_offsets, tm_fuse_match *fuse, tm_fuse_match *fwd,
                            int32_t *fwd_offsets, float *points, uint8_t *point_ok);
/* Counters of a server since its start (admission by memory and eviction made visible).
 *   submitted, admitted, completed, failed   requests (failed: completed with an error)
 *   batches                                  launches of a batch (search + fusion)
 *   deferrals                                admission rounds that left requests waiting
 *                                            for a store slot (admission by memory)
 *   evicted                                  keyframes the server removed (evict_after)
 *   peak_pending                             most requests queued at once
 *   peak_inflight                            most batches on the GPU at once
 *   peak_store_slots                         most keyframe slots in use at once (whole store)
 *   store_slot_limit                         slots the context's budget allows (-1: free memory
 *                                            decides) */
typedef struct {
    int64_t submitted, admitted, completed, failed, batches, deferrals, evicted;
    int32_t peak_pending, peak_inflight, peak_store_slots, store_slot_limit;
} tm_server_stats;
tm_status tm_server_get_stats(tm_server *srv, tm_server_stats *out);
/* Drains the queue, stops the thread, frees the server. */
tm_status tm_server_stop(tm_server *srv);

/* Monotonic clock used by the server (seconds). */
double tm_now(void);

/* ---------------------------------------------------------------------------- no allocation
 * The paper has no counterpart to this call.  It is for callers that cannot allocate device
 * memory: code under an allocator that must not grow (a fixed memory budget), a real-time
 * loop that forbids allocation after start-up (an allocation may block or synchronise the
 * device), or a host without a tm_ctx (whose keyframe store allocates).
 *
 * Correspondence search of one keyframe pair, with the same results as tm_search_
 * triangulation(q, [t]).  It allocates nothing: its scratch -- both keyframes in node order
 * with their projection grids, the per-pair arrays and the counters -- lives in one fixed
 * array inside the library (about 256 KB, held by every GPU that loads the library until
 * the process exits).
 *   q, t       keyframes of at most TM_NOALLOC_MAX_KP keypoints each; their arrays must be
 *              memory of the current device (or managed memory), desc 16-byte, xy 8-byte,
 *              angle and node 4-byte aligned (Tcw is read from the struct); larger keyframes,
 *              host or another device's memory and misaligned arrays are rejected with
 *              TM_ERR_INVALID_ARG before any work
 *   params     NULL = defaults; mode, dense_min and baseline_min_ratio are ignored (this call
 *              always runs the plain per-pair kernels and has no median scene depth), the
 *              other fields are checked as by tm_search_triangulation
 *   q_free, t_free  device [n] or NULL
 *   out        device tm_match [q->n] (4-byte aligned), matches sorted by q_idx
 *   n_out      device uint32 (4-byte aligned): number of matches
 *   n_comparisons   device uint64 (8-byte aligned) or NULL
 * Asynchronous on `stream` (NULL: the legacy default stream): results are valid once the
 * stream reaches this call, and the inputs must stay valid until then.  The first call on a
 * device looks up the array's device address (once per device, with that device current)
 * and keeps it for the life of the process: make that first call before any stream capture,
 * and do not reset the device (cudaDeviceReset) while the library is loaded.  Every call uses
 * the same array and leaves its contents behind (each call clears what must start at zero):
 * calls whose work may overlap on the GPU -- on different streams or threads -- race with one
 * another; calls on one stream run one after the other. */
#define TM_NOALLOC_MAX_KP 2048
tm_status tm_search_pair_noalloc(const tm_camera *cam, const tm_keyframe_view *q,
                                 const tm_keyframe_view *t, const tm_search_params *params,
                                 const uint8_t *q_free, const uint8_t *t_free, tm_match *out,
                                 uint32_t *n_out, uint64_t *n_comparisons, void *stream);

#ifdef __cplusplus
}
#endif
#endif
