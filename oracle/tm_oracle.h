/*
 * Oracle for the local-mapping correspondence search and map-point fusion search.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct CPU definition of
 * what the GPU library computes.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the library itself never does.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it follows (TurboMap, Hosseininejad et al.):
 *   - Sec. IV-C  Keypoint Correspondence Search: for each keypoint of the new keyframe,
 *                compare descriptors against the candidate keypoints of one neighbouring
 *                keyframe and validate candidates with the epipolar constraint.  Search is
 *                decoupled from triangulation, so every neighbour is searched independently.
 *   - Sec. IV-D  Map-point Fusion: for each map point and one keyframe, find the most similar
 *                keypoint by projection and descriptor distance; merging is deferred.
 * The paper does not spell out the matching rules; the readings taken here (BoW-node
 * buckets, Hamming <= 50, ratio 0.6, chi2 3.84 sigma^2 epipolar gate, one match per target,
 * 30-bin rotation histogram keeping the top three bins, radius 3*scale projection window,
 * chi2 5.99 sigma^2 reprojection gate) are listed with every other reading in the design
 * notes of the repository.
 *
 * Built with -O2 -ffp-contract=off -fno-fast-math: no fused multiply-add, IEEE float.
 * Floating-point decisions (the gates) are taken in float32, the precision of the GPU path;
 * the fundamental matrix is formed in float64 and rounded to float32.
 */
#ifndef TM_ORACLE_H
#define TM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
} orc_camera;

typedef struct {
    int32_t n;
    const uint8_t *desc;    /* [n][32] */
    const float *xy;        /* [n][2]  */
    const float *angle;     /* [n] degrees */
    const uint8_t *level;   /* [n] 0..7 */
    const uint32_t *node;   /* [n] */
    double Tcw[12];         /* row-major 3x4, world -> camera */
} orc_keyframe;

typedef struct {
    int32_t hamming_max;    /* accept only best <= hamming_max                (50)   */
    int32_t ratio_num;      /* accept only ratio_den*best < ratio_num*second  (3)    */
    int32_t ratio_den;      /*   ratio test disabled when ratio_num == 0      (5)    */
    float epi_chi2;         /* epipolar gate: dist^2 < epi_chi2*sigma^2(level) (3.84) */
    int32_t epipolar;       /* 1: apply the epipolar gate                            */
    int32_t resolve;        /* 1: keep one match per target keypoint                  */
    int32_t rot_filter;     /* 1: apply the rotation-histogram filter                 */
    /* ORB-family variants (off by default) */
    float epipole_px;       /* > 0: drop a candidate whose squared distance to the epipole
                               (Q's centre projected into T) is below
                               epipole_px^2 * scale(level of the candidate)              */
    int32_t rot_mode;       /* 0: 30 bins of 12 degrees, floor(rot / 12);
                               1: ORB-family bins round(rot * (1/30)), 30 -> 0            */
    float baseline_min_ratio; /* > 0: skip the pair when |C_Q - C_T| / t_median_depth is
                               below it (t_median_depth > 0 only)                          */
    float t_median_depth;   /* the neighbour's median scene depth (0 = unknown)            */
} orc_search_params;

typedef struct {
    float chi2;             /* reprojection gate e^2 <= chi2*sigma^2(level)  (5.99) */
    int32_t hamming_max;    /* (50) */
    float radius_scale;     /* window half-width = radius_scale*scale[level] (3.0) */
} orc_fuse_params;

/* The epipole in T: Q's camera centre C_Q = -R_Q^T t_Q projected into T (float64, rounded
 * to float32); +-inf or NaN when C_Q lies in T's principal plane. */
void orc_epipole(const orc_camera *cam, const double Tcw_q[12], const double Tcw_t[12], float e[2]);
/* Rotation bin of a match (rot_mode as in orc_search_params). */
int orc_rot_bin_mode(float angle_q, float angle_t, int mode);

/* Triangulation of matches and their acceptance as new map points (Sec. III, Map Point
 * Creation: sufficient parallax, positive depth, low reprojection error, scale consistency). */
typedef struct {
    double cos_parallax_max;  /* accept only 0 < cos(angle between the rays) < this (0.9998) */
    double chi2;              /* reprojection error^2 <= chi2 * sigma^2(level), each view (5.991) */
    double ratio_factor;      /* scale consistency factor (1.5 * 1.2)                       */
} orc_tri_params;
/* For n matches (q_idx[k] of Q, t_idx[k] of T): xyz[3k..3k+2] the triangulated point
 * (float32; 0 when rejected), ok[k] = 1 when every constraint holds. */
void orc_triangulate(const orc_camera *cam, const orc_keyframe *Q, const orc_keyframe *T,
                     int64_t n, const int32_t *q_idx, const int32_t *t_idx,
                     const orc_tri_params *p, float *xyz, uint8_t *ok);

/* F (float32, row-major 3x3) with x_Q^T F x_T = 0 for corresponding pixels. */
void orc_fundamental(const orc_camera *cam, const double Tcw_q[12], const double Tcw_t[12],
                     float F[9]);

/* Search one (Q, T) pair.  free_q / free_t may be NULL (all free).  Writes up to `cap`
 * matches (q, t, dist), sorted by q, and returns the number of matches (which may exceed
 * cap; nothing past cap is written).  *n_comparisons = number of (i, j) with free i, free j
 * and equal node, i.e. the descriptor comparisons the method must perform. */
int64_t orc_search_pair(const orc_camera *cam, const orc_keyframe *Q, const orc_keyframe *T,
                        const uint8_t *free_q, const uint8_t *free_t,
                        const orc_search_params *p, int32_t *out_q, int32_t *out_t,
                        int32_t *out_d, int64_t cap, int64_t *n_comparisons);

/* Fuse n map points into keyframe T.  skip may be NULL.  Writes (mp, kp, dist) sorted by mp
 * and returns the count; *n_comparisons = number of (map point, keypoint) pairs inside the
 * projection window at an admissible level. */
int64_t orc_fuse(const orc_camera *cam, const orc_keyframe *T, int32_t n, const float *pos,
                 const float *normal, const uint8_t *desc, const float *min_dist,
                 const float *max_dist, const uint8_t *skip, const orc_fuse_params *p,
                 int32_t *out_m, int32_t *out_k, int32_t *out_d, int64_t cap,
                 int64_t *n_comparisons);

#ifdef __cplusplus
}
#endif
#endif
