/*
 * Oracle: plain CPU definition of the correspondence search (Sec. IV-C) and the fusion
 * search (Sec. IV-D).  TEST INFRASTRUCTURE ONLY -- see tm_oracle.h.
 *
 * Everything is a direct nested loop over (query keypoint, target keypoint): no buckets,
 * no grids, no sorting, no parallelism.  The BoW-node condition is a predicate inside the
 * loop, the projection window is a predicate inside the loop.
 */
#include "tm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LEVELS 8
#define ORC_BINS 30

/* Pyramid tables in float32: scale[0] = 1, scale[l] = scale[l-1] * 1.2 (repeated
 * multiplication, no pow). */
static void orc_scales(float scale[ORC_LEVELS], float sigma2[ORC_LEVELS]) {
    scale[0] = 1.0f;
    for (int l = 1; l < ORC_LEVELS; ++l) scale[l] = scale[l - 1] * 1.2f;
    for (int l = 0; l < ORC_LEVELS; ++l) sigma2[l] = scale[l] * scale[l];
}

/* Hamming distance of two 256-bit descriptors: count of differing bits, bit by bit. */
static int orc_hamming(const uint8_t *a, const uint8_t *b) {
    int d = 0;
    for (int byte = 0; byte < 32; ++byte) {
        uint8_t x = (uint8_t)(a[byte] ^ b[byte]);
        for (int bit = 0; bit < 8; ++bit) d += (x >> bit) & 1u;
    }
    return d;
}

/* 3x3 product C = A*B, each entry summed k = 0, 1, 2 left to right, float64. */
static void orc_mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = A[r * 3 + 0] * B[0 * 3 + c];
            s = s + A[r * 3 + 1] * B[1 * 3 + c];
            s = s + A[r * 3 + 2] * B[2 * 3 + c];
            C[r * 3 + c] = s;
        }
}

/* Fundamental matrix between the new keyframe Q and a neighbour T (Sec. IV-C's epipolar
 * validation).  With world->camera poses X_Q = R_Q X + t_Q and X_T = R_T X + t_T, the
 * relative motion T -> Q is R = R_Q R_T^T, t = t_Q - R t_T, the essential matrix is
 * E = [t]x R and F = K^-T E K^-1, so that x_Q^T F x_T = 0.  All float64, products
 * evaluated left to right as ((K^-T [t]x) R) K^-1, then each entry rounded to float32. */
void orc_fundamental(const orc_camera *cam, const double Tq[12], const double Tt[12],
                     float F[9]) {
    double Rq[9], Rt[9], tq[3], tt[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            Rq[r * 3 + c] = Tq[r * 4 + c];
            Rt[r * 3 + c] = Tt[r * 4 + c];
        }
        tq[r] = Tq[r * 4 + 3];
        tt[r] = Tt[r * 4 + 3];
    }
    double RtT[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) RtT[r * 3 + c] = Rt[c * 3 + r];
    double R[9];
    orc_mat3_mul(Rq, RtT, R);
    double t[3];
    for (int r = 0; r < 3; ++r) {
        double s = R[r * 3 + 0] * tt[0];
        s = s + R[r * 3 + 1] * tt[1];
        s = s + R[r * 3 + 2] * tt[2];
        t[r] = tq[r] - s;
    }
    const double tx[9] = {0.0, -t[2], t[1],
                          t[2], 0.0, -t[0],
                          -t[1], t[0], 0.0};
    const double Kinv[9] = {1.0 / cam->fx, 0.0, -cam->cx / cam->fx,
                            0.0, 1.0 / cam->fy, -cam->cy / cam->fy,
                            0.0, 0.0, 1.0};
    double KinvT[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) KinvT[r * 3 + c] = Kinv[c * 3 + r];
    double A[9], B[9], Fd[9];
    orc_mat3_mul(KinvT, tx, A);
    orc_mat3_mul(A, R, B);
    orc_mat3_mul(B, Kinv, Fd);
    for (int k = 0; k < 9; ++k) F[k] = (float)Fd[k];
}

/* Epipolar gate: squared distance of x_T to the epipolar line l = F^T x_Q of query x_Q,
 * below chi2 * sigma^2(level of the target keypoint).  Division-free form
 * num^2 < thr * (a^2 + b^2), float32, evaluated in the stated order. */
static int orc_epipolar_ok(const float F[9], float xq, float yq, float xt, float yt,
                           float thr) {
    float a = (xq * F[0] + yq * F[3]) + F[6];
    float b = (xq * F[1] + yq * F[4]) + F[7];
    float c = (xq * F[2] + yq * F[5]) + F[8];
    float num = (a * xt + b * yt) + c;
    float den = a * a + b * b;
    if (!(den > 0.0f)) return 0;
    return num * num < thr * den;
}

/* Rotation-histogram bin of an accepted match over the orientation difference
 * angle_Q - angle_T wrapped into [0, 360): mode 0, 30 bins of 12 degrees; mode 1, the
 * ORB-family binning, the nearest integer of rot * (1/30) (float32 factor; halves away from
 * zero), 30 folded to 0, so that only bins 0..12 occur. */
int orc_rot_bin_mode(float angle_q, float angle_t, int mode) {
    float rot = angle_q - angle_t;
    if (rot < 0.0f) rot += 360.0f;
    int bin = mode == 1 ? (int)roundf(rot * (1.0f / 30.0f)) : (int)floorf(rot / 12.0f);
    if (bin >= ORC_BINS) bin = 0;
    return bin;
}

/* The epipole in T, the image of Q's camera centre: C_Q = -R_Q^T t_Q, C = R_T C_Q + t_T,
 * e = (fx * (C_x / C_z) + cx, fy * (C_y / C_z) + cy), all float64, sums left to right,
 * rounded to float32 at the end. */
void orc_epipole(const orc_camera *cam, const double Tq[12], const double Tt[12], float e[2]) {
    double cq[3], c[3];
    for (int k = 0; k < 3; ++k) {
        double s = Tq[0 * 4 + k] * Tq[0 * 4 + 3];
        s = s + Tq[1 * 4 + k] * Tq[1 * 4 + 3];
        s = s + Tq[2 * 4 + k] * Tq[2 * 4 + 3];
        cq[k] = -s;
    }
    for (int r = 0; r < 3; ++r) {
        double s = Tt[r * 4 + 0] * cq[0];
        s = s + Tt[r * 4 + 1] * cq[1];
        s = s + Tt[r * 4 + 2] * cq[2];
        c[r] = s + Tt[r * 4 + 3];
    }
    e[0] = (float)(cam->fx * (c[0] / c[2]) + cam->cx);
    e[1] = (float)(cam->fy * (c[1] / c[2]) + cam->cy);
}

int64_t orc_search_pair(const orc_camera *cam, const orc_keyframe *Q, const orc_keyframe *T,
                        const uint8_t *free_q, const uint8_t *free_t,
                        const orc_search_params *p, int32_t *out_q, int32_t *out_t,
                        int32_t *out_d, int64_t cap, int64_t *n_comparisons) {
    float scale[ORC_LEVELS], sigma2[ORC_LEVELS], thr[ORC_LEVELS];
    orc_scales(scale, sigma2);
    for (int l = 0; l < ORC_LEVELS; ++l) thr[l] = p->epi_chi2 * sigma2[l];
    /* ORB-family pair-baseline skip: with the neighbour's median scene depth known, a pair
     * whose baseline |C_Q - C_T| (camera centres C = -R^T t, float64) is below
     * baseline_min_ratio * depth (as baseline / depth < ratio, float64) is not searched. */
    if (p->baseline_min_ratio > 0.0f && p->t_median_depth > 0.0f) {
        double c[2][3];
        const double *P[2] = {Q->Tcw, T->Tcw};
        for (int v = 0; v < 2; ++v)
            for (int k = 0; k < 3; ++k) {
                double s = P[v][0 * 4 + k] * P[v][0 * 4 + 3];
                s = s + P[v][1 * 4 + k] * P[v][1 * 4 + 3];
                s = s + P[v][2 * 4 + k] * P[v][2 * 4 + 3];
                c[v][k] = -s;
            }
        const double dx = c[0][0] - c[1][0], dy = c[0][1] - c[1][1], dz = c[0][2] - c[1][2];
        const double base = sqrt(dx * dx + dy * dy + dz * dz);
        if (base / (double)p->t_median_depth < (double)p->baseline_min_ratio) {
            if (n_comparisons) *n_comparisons = 0;
            return 0;
        }
    }
    float F[9];
    orc_fundamental(cam, Q->Tcw, T->Tcw, F);
    /* ORB-family epipole rejection: a candidate whose squared distance to the epipole is
     * below epipole_px^2 * scale(level) (float32, (dx*dx) + (dy*dy)) is dropped after its
     * distance is computed, like a failed epipolar gate. */
    float ep[2] = {0.0f, 0.0f}, thr_e[ORC_LEVELS];
    const int use_ep = p->epipole_px > 0.0f;
    if (use_ep) orc_epipole(cam, Q->Tcw, T->Tcw, ep);
    for (int l = 0; l < ORC_LEVELS; ++l) thr_e[l] = (p->epipole_px * p->epipole_px) * scale[l];

    const int nq = Q->n, nt = T->n;
    int *acc_t = (int *)malloc(sizeof(int) * (size_t)(nq > 0 ? nq : 1));
    int *acc_d = (int *)malloc(sizeof(int) * (size_t)(nq > 0 ? nq : 1));
    int64_t comparisons = 0;

    /* Step 1: best / second-best over the candidates of each free query keypoint.
     * A candidate is a free target keypoint with the same BoW node that passes the
     * epipolar gate.  best = smallest distance, ties to the lowest target index;
     * second = second-smallest distance of the multiset (equal to best on a tie). */
    for (int i = 0; i < nq; ++i) {
        acc_t[i] = -1;
        acc_d[i] = 0;
        if (free_q && !free_q[i]) continue;
        int best = 0x7fffffff, second = 0x7fffffff, best_j = -1;
        for (int j = 0; j < nt; ++j) {
            if (free_t && !free_t[j]) continue;
            if (Q->node[i] != T->node[j]) continue;
            comparisons++;
            int d = orc_hamming(Q->desc + 32 * (size_t)i, T->desc + 32 * (size_t)j);
            if (p->epipolar &&
                !orc_epipolar_ok(F, Q->xy[2 * i], Q->xy[2 * i + 1], T->xy[2 * j],
                                 T->xy[2 * j + 1], thr[T->level[j]]))
                continue;
            if (use_ep) {
                const float dx = ep[0] - T->xy[2 * j], dy = ep[1] - T->xy[2 * j + 1];
                if (dx * dx + dy * dy < thr_e[T->level[j]]) continue;
            }
            if (d < best) {
                second = best;
                best = d;
                best_j = j;
            } else if (d < second) {
                second = d;
            }
        }
        if (best_j < 0) continue;
        if (best > p->hamming_max) continue;
        /* ratio test best < 0.6 * second in the exact integer form 5*best < 3*second;
         * with a single candidate there is no second and the test passes. */
        if (p->ratio_num != 0 && second != 0x7fffffff &&
            !((int64_t)p->ratio_den * best < (int64_t)p->ratio_num * second))
            continue;
        acc_t[i] = best_j;
        acc_d[i] = best;
    }

    /* Step 2: one match per target keypoint.  For every target j the accepted query with
     * the lowest (distance, query index) keeps it; the others are dropped, not re-matched. */
    if (p->resolve) {
        for (int j = 0; j < nt; ++j) {
            int win = -1;
            for (int i = 0; i < nq; ++i) {
                if (acc_t[i] != j) continue;
                if (win < 0 || acc_d[i] < acc_d[win]) win = i;
            }
            for (int i = 0; i < nq; ++i)
                if (acc_t[i] == j && i != win) acc_t[i] = -1;
        }
    }

    /* Step 3: rotation consistency.  Histogram the orientation difference of the kept
     * matches into 30 bins, take the three most populated bins (ties to the lower bin,
     * empty bins never taken), drop the 2nd and 3rd when they hold less than a tenth of
     * the largest (integer form 10*count < max), keep only matches in the taken bins. */
    if (p->rot_filter) {
        int hist[ORC_BINS];
        memset(hist, 0, sizeof hist);
        for (int i = 0; i < nq; ++i)
            if (acc_t[i] >= 0) hist[orc_rot_bin_mode(Q->angle[i], T->angle[acc_t[i]], p->rot_mode)]++;
        int top[3] = {-1, -1, -1};
        for (int r = 0; r < 3; ++r) {
            int bestb = -1;
            for (int b = 0; b < ORC_BINS; ++b) {
                if (hist[b] == 0) continue;
                if (b == top[0] || b == top[1]) continue;
                if (bestb < 0 || hist[b] > hist[bestb]) bestb = b;
            }
            top[r] = bestb;
        }
        if (top[0] >= 0) {
            int mx = hist[top[0]];
            for (int r = 1; r < 3; ++r)
                if (top[r] >= 0 && 10 * hist[top[r]] < mx) top[r] = -1;
        }
        for (int i = 0; i < nq; ++i) {
            if (acc_t[i] < 0) continue;
            int b = orc_rot_bin_mode(Q->angle[i], T->angle[acc_t[i]], p->rot_mode);
            if (b != top[0] && b != top[1] && b != top[2]) acc_t[i] = -1;
        }
    }

    int64_t count = 0;
    for (int i = 0; i < nq; ++i) {
        if (acc_t[i] < 0) continue;
        if (count < cap) {
            out_q[count] = i;
            out_t[count] = acc_t[i];
            out_d[count] = acc_d[i];
        }
        count++;
    }
    free(acc_t);
    free(acc_d);
    if (n_comparisons) *n_comparisons = comparisons;
    return count;
}

int64_t orc_fuse(const orc_camera *cam, const orc_keyframe *T, int32_t n, const float *pos,
                 const float *normal, const uint8_t *desc, const float *min_dist,
                 const float *max_dist, const uint8_t *skip, const orc_fuse_params *p,
                 int32_t *out_m, int32_t *out_k, int32_t *out_d, int64_t cap,
                 int64_t *n_comparisons) {
    float scale[ORC_LEVELS], sigma2[ORC_LEVELS], thr[ORC_LEVELS];
    orc_scales(scale, sigma2);
    for (int l = 0; l < ORC_LEVELS; ++l) thr[l] = p->chi2 * sigma2[l];

    /* Pose of the target keyframe in float32, and its camera centre O = -R^T t formed in
     * float64 and rounded. */
    float R[9], t[3], O[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[r * 3 + c] = (float)T->Tcw[r * 4 + c];
        t[r] = (float)T->Tcw[r * 4 + 3];
    }
    for (int c = 0; c < 3; ++c) {
        double s = T->Tcw[0 * 4 + c] * T->Tcw[0 * 4 + 3];
        s = s + T->Tcw[1 * 4 + c] * T->Tcw[1 * 4 + 3];
        s = s + T->Tcw[2 * 4 + c] * T->Tcw[2 * 4 + 3];
        O[c] = (float)(-s);
    }
    const float fx = (float)cam->fx, fy = (float)cam->fy;
    const float cx = (float)cam->cx, cy = (float)cam->cy;
    const float W = (float)cam->width, H = (float)cam->height;

    int64_t count = 0, comparisons = 0;
    for (int m = 0; m < n; ++m) {
        if (skip && skip[m]) continue;
        const float X = pos[3 * m], Y = pos[3 * m + 1], Z = pos[3 * m + 2];
        /* projection into the target keyframe */
        float xc = ((R[0] * X + R[1] * Y) + R[2] * Z) + t[0];
        float yc = ((R[3] * X + R[4] * Y) + R[5] * Z) + t[1];
        float zc = ((R[6] * X + R[7] * Y) + R[8] * Z) + t[2];
        if (!(zc > 0.0f)) continue;
        float x = xc / zc, y = yc / zc;
        float u = fx * x + cx, v = fy * y + cy;
        if (!(u >= 0.0f && u < W && v >= 0.0f && v < H)) continue;
        /* distance and viewing-angle gates */
        float pox = X - O[0], poy = Y - O[1], poz = Z - O[2];
        float dist = sqrtf((pox * pox + poy * poy) + poz * poz);
        if (dist < min_dist[m] || dist > max_dist[m]) continue;
        float cosv = (pox * normal[3 * m] + poy * normal[3 * m + 1]) + poz * normal[3 * m + 2];
        if (cosv < 0.5f * dist) continue;
        /* predicted pyramid level: smallest l with dist * scale[l] >= maxDist, else 7 */
        int pl = ORC_LEVELS - 1;
        for (int l = 0; l < ORC_LEVELS; ++l)
            if (dist * scale[l] >= max_dist[m]) {
                pl = l;
                break;
            }
        float r = p->radius_scale * scale[pl];
        /* best keypoint in the window at level pl-1 or pl */
        int best = 0x7fffffff, best_j = -1;
        for (int j = 0; j < T->n; ++j) {
            int lv = T->level[j];
            if (lv != pl && lv != pl - 1) continue;
            float xt = T->xy[2 * j], yt = T->xy[2 * j + 1];
            if (!(fabsf(xt - u) < r && fabsf(yt - v) < r)) continue;
            comparisons++;
            float ex = u - xt, ey = v - yt;
            if (!((ex * ex + ey * ey) <= thr[lv])) continue;
            int d = orc_hamming(desc + 32 * (size_t)m, T->desc + 32 * (size_t)j);
            if (d < best) {
                best = d;
                best_j = j;
            }
        }
        if (best_j < 0 || best > p->hamming_max) continue;
        if (count < cap) {
            out_m[count] = m;
            out_k[count] = best_j;
            out_d[count] = best;
        }
        count++;
    }
    if (n_comparisons) *n_comparisons = comparisons;
    return count;
}


/* ------------------------------------------------------------------ triangulation
 * Map Point Creation after the search (Sec. III): each match is triangulated and kept as a
 * new map point only if the two views see it with sufficient parallax, in front of both
 * cameras, with a low reprojection error in each view, and at consistent scales.  The paper
 * gives the constraints, not their formulas; the readings, all float32 (a pose's R and t
 * rounded from float64, its centre O = -R^T t formed in float64 and rounded; dot products
 * (x*x' + y*y') + z*z'):
 *   normalized coordinates  xn = (u - cx) / fx, yn = (v - cy) / fy;
 *   rays in the world frame r = R^T (xn, yn, 1); parallax cos = (r1.r2) / (|r1| |r2|),
 *     kept iff 0 < cos < cos_parallax_max;
 *   the point: the midpoint of the common perpendicular of the rays O1 + s r1, O2 + t r2:
 *     w = O1 - O2, a = r1.r1, b = r1.r2, c = r2.r2, d = r1.w, e = r2.w, den = a c - b b
 *     (rejected if not > 0), s = (b e - c d) / den, t = (a e - b d) / den,
 *     X = ((O1 + s r1) + (O2 + t r2)) * 0.5;
 *   depth z = R_3 X + t_3 > 0 in both views;
 *   reprojection (fx x/z + cx - u)^2 + (fy y/z + cy - v)^2 <= chi2 * sigma^2(level), each view;
 *   scale: d_i = |X - O_i|, ratio_dist = d2 / d1, ratio_octave = s(l1) / s(l2);
 *     rejected if ratio_dist * f < ratio_octave or ratio_dist > ratio_octave * f. */
typedef struct { float R[9], t[3], O[3]; } orc_view;

static void orc_view_of(const double Tcw[12], orc_view *v) {
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) v->R[r * 3 + c] = (float)Tcw[r * 4 + c];
        v->t[r] = (float)Tcw[r * 4 + 3];
    }
    for (int k = 0; k < 3; ++k) {
        double s = Tcw[0 * 4 + k] * Tcw[0 * 4 + 3];
        s = s + Tcw[1 * 4 + k] * Tcw[1 * 4 + 3];
        s = s + Tcw[2 * 4 + k] * Tcw[2 * 4 + 3];
        v->O[k] = (float)(-s);
    }
}

static float orc_dot3(const float *a, const float *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

/* depth and reprojection test of X in one view */
static int orc_view_ok(const orc_camera *cam, const orc_view *v, const float X[3], float u, float vv,
                       float thr) {
    float c[3];
    for (int r = 0; r < 3; ++r) c[r] = ((v->R[r * 3 + 0] * X[0] + v->R[r * 3 + 1] * X[1]) + v->R[r * 3 + 2] * X[2]) + v->t[r];
    if (!(c[2] > 0.0f)) return 0;
    const float eu = ((float)cam->fx * (c[0] / c[2]) + (float)cam->cx) - u;
    const float ev = ((float)cam->fy * (c[1] / c[2]) + (float)cam->cy) - vv;
    return eu * eu + ev * ev <= thr;
}

void orc_triangulate(const orc_camera *cam, const orc_keyframe *Q, const orc_keyframe *T,
                     int64_t n, const int32_t *q_idx, const int32_t *t_idx,
                     const orc_tri_params *p, float *xyz, uint8_t *ok) {
    float scale[ORC_LEVELS], sigma2[ORC_LEVELS];
    orc_scales(scale, sigma2);
    orc_view V[2];
    orc_view_of(Q->Tcw, &V[0]);
    orc_view_of(T->Tcw, &V[1]);
    const float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    const float cos_max = (float)p->cos_parallax_max, chi2 = (float)p->chi2, f = (float)p->ratio_factor;
    for (int64_t k = 0; k < n; ++k) {
        const orc_keyframe *kf[2] = {Q, T};
        const int idx[2] = {q_idx[k], t_idx[k]};
        float u[2], vv[2], ray[2][3];
        int lev[2];
        for (int s = 0; s < 2; ++s) {
            u[s] = kf[s]->xy[2 * idx[s]];
            vv[s] = kf[s]->xy[2 * idx[s] + 1];
            lev[s] = kf[s]->level[idx[s]];
            const float xn = (u[s] - cx) / fx, yn = (vv[s] - cy) / fy;
            for (int c = 0; c < 3; ++c)
                ray[s][c] = (V[s].R[0 * 3 + c] * xn + V[s].R[1 * 3 + c] * yn) + V[s].R[2 * 3 + c];
        }
        xyz[3 * k] = xyz[3 * k + 1] = xyz[3 * k + 2] = 0.0f;
        ok[k] = 0;
        const float a = orc_dot3(ray[0], ray[0]), b = orc_dot3(ray[0], ray[1]), c2 = orc_dot3(ray[1], ray[1]);
        const float cosp = b / (sqrtf(a) * sqrtf(c2));
        if (!(cosp > 0.0f && cosp < cos_max)) continue;
        float w[3];
        for (int q = 0; q < 3; ++q) w[q] = V[0].O[q] - V[1].O[q];
        const float d = orc_dot3(ray[0], w), e = orc_dot3(ray[1], w);
        const float den = a * c2 - b * b;
        if (!(den > 0.0f)) continue;
        const float s1 = (b * e - c2 * d) / den, s2 = (a * e - b * d) / den;
        float X[3];
        for (int q = 0; q < 3; ++q) X[q] = ((V[0].O[q] + s1 * ray[0][q]) + (V[1].O[q] + s2 * ray[1][q])) * 0.5f;
        if (!orc_view_ok(cam, &V[0], X, u[0], vv[0], chi2 * sigma2[lev[0]])) continue;
        if (!orc_view_ok(cam, &V[1], X, u[1], vv[1], chi2 * sigma2[lev[1]])) continue;
        float dist[2];
        for (int s = 0; s < 2; ++s) {
            float dv[3];
            for (int q = 0; q < 3; ++q) dv[q] = X[q] - V[s].O[q];
            dist[s] = sqrtf(orc_dot3(dv, dv));
        }
        if (dist[0] == 0.0f || dist[1] == 0.0f) continue;
        const float ratio_dist = dist[1] / dist[0];
        const float ratio_octave = scale[lev[0]] / scale[lev[1]];
        if (ratio_dist * f < ratio_octave || ratio_dist > ratio_octave * f) continue;
        for (int q = 0; q < 3; ++q) xyz[3 * k + q] = X[q];
        ok[k] = 1;
    }
}
