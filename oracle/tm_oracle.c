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
 * gives the constraints, not their formulas; the readings (all float64, sums left to right):
 *   normalized coordinates  xn = (u - cx) / fx, yn = (v - cy) / fy;
 *   rays in the world frame r = R^T (xn, yn, 1); parallax cos = (r1.r2) / (|r1| |r2|),
 *     kept iff 0 < cos < cos_parallax_max;
 *   linear triangulation: with P = [R | t] each view gives the rows xn P_3 - P_1 and
 *     yn P_3 - P_2 of A (4 x 4); X solves the least-squares problem A_{:,0:3} X = -A_{:,3}
 *     through its normal equations (A3^T A3) X = A3^T b, by Cramer's rule (det 0: rejected);
 *   depth z = R_3 X + t_3 > 0 in both views;
 *   reprojection (fx x/z + cx - u)^2 + (fy y/z + cy - v)^2 <= chi2 * sigma^2(level), each view;
 *   scale: d_i = |X - O_i| (O = -R^T t), ratio_dist = d2 / d1, ratio_octave = s(l1) / s(l2);
 *     rejected if ratio_dist * f < ratio_octave or ratio_dist > ratio_octave * f. */
static double orc_det3(const double m[9]) {
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

/* One view: R (row-major 3x3), t, its camera centre O, and the pixel's normalized
 * coordinates and world ray. */
typedef struct { double R[9], t[3], O[3]; } orc_view;

static void orc_view_of(const double Tcw[12], orc_view *v) {
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) v->R[r * 3 + c] = Tcw[r * 4 + c];
        v->t[r] = Tcw[r * 4 + 3];
    }
    for (int k = 0; k < 3; ++k) {
        double s = v->R[0 * 3 + k] * v->t[0];
        s = s + v->R[1 * 3 + k] * v->t[1];
        s = s + v->R[2 * 3 + k] * v->t[2];
        v->O[k] = -s;
    }
}

/* depth and reprojection test of X in one view */
static int orc_view_ok(const orc_camera *cam, const orc_view *v, const double X[3], double u,
                       double vv, double thr) {
    double c[3];
    for (int r = 0; r < 3; ++r) {
        double s = v->R[r * 3 + 0] * X[0];
        s = s + v->R[r * 3 + 1] * X[1];
        s = s + v->R[r * 3 + 2] * X[2];
        c[r] = s + v->t[r];
    }
    if (!(c[2] > 0.0)) return 0;
    const double eu = (cam->fx * (c[0] / c[2]) + cam->cx) - u;
    const double ev = (cam->fy * (c[1] / c[2]) + cam->cy) - vv;
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
    for (int64_t k = 0; k < n; ++k) {
        const orc_keyframe *kf[2] = {Q, T};
        const int idx[2] = {q_idx[k], t_idx[k]};
        double u[2], vv[2], xn[2], yn[2], ray[2][3], rn[2];
        int lev[2];
        for (int s = 0; s < 2; ++s) {
            u[s] = kf[s]->xy[2 * idx[s]];
            vv[s] = kf[s]->xy[2 * idx[s] + 1];
            lev[s] = kf[s]->level[idx[s]];
            xn[s] = (u[s] - cam->cx) / cam->fx;
            yn[s] = (vv[s] - cam->cy) / cam->fy;
            for (int c = 0; c < 3; ++c) {
                double r = V[s].R[0 * 3 + c] * xn[s];
                r = r + V[s].R[1 * 3 + c] * yn[s];
                ray[s][c] = r + V[s].R[2 * 3 + c];
            }
            rn[s] = sqrt(ray[s][0] * ray[s][0] + ray[s][1] * ray[s][1] + ray[s][2] * ray[s][2]);
        }
        xyz[3 * k] = xyz[3 * k + 1] = xyz[3 * k + 2] = 0.0f;
        ok[k] = 0;
        const double cosp = (ray[0][0] * ray[1][0] + ray[0][1] * ray[1][1] + ray[0][2] * ray[1][2]) / (rn[0] * rn[1]);
        if (!(cosp > 0.0 && cosp < p->cos_parallax_max)) continue;
        /* rows xn P_3 - P_1, yn P_3 - P_2 of each view, P = [R | t] */
        double A[4][4];
        for (int s = 0; s < 2; ++s)
            for (int c = 0; c < 4; ++c) {
                const double p3 = c < 3 ? V[s].R[2 * 3 + c] : V[s].t[2];
                const double p1 = c < 3 ? V[s].R[0 * 3 + c] : V[s].t[0];
                const double p2 = c < 3 ? V[s].R[1 * 3 + c] : V[s].t[1];
                A[2 * s][c] = xn[s] * p3 - p1;
                A[2 * s + 1][c] = yn[s] * p3 - p2;
            }
        double N[9], g[3];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) {
                double s = A[0][r] * A[0][c];
                for (int q = 1; q < 4; ++q) s = s + A[q][r] * A[q][c];
                N[r * 3 + c] = s;
            }
            double s = A[0][r] * -A[0][3];
            for (int q = 1; q < 4; ++q) s = s + A[q][r] * -A[q][3];
            g[r] = s;
        }
        const double det = orc_det3(N);
        if (det == 0.0) continue;
        double X[3];
        for (int c = 0; c < 3; ++c) {
            double M[9];
            for (int q = 0; q < 9; ++q) M[q] = N[q];
            for (int r = 0; r < 3; ++r) M[r * 3 + c] = g[r];
            X[c] = orc_det3(M) / det;
        }
        if (!orc_view_ok(cam, &V[0], X, u[0], vv[0], p->chi2 * (double)sigma2[lev[0]])) continue;
        if (!orc_view_ok(cam, &V[1], X, u[1], vv[1], p->chi2 * (double)sigma2[lev[1]])) continue;
        double d[2];
        for (int s = 0; s < 2; ++s) {
            const double dx = X[0] - V[s].O[0], dy = X[1] - V[s].O[1], dz = X[2] - V[s].O[2];
            d[s] = sqrt(dx * dx + dy * dy + dz * dz);
        }
        if (d[0] == 0.0 || d[1] == 0.0) continue;
        const double ratio_dist = d[1] / d[0];
        const double ratio_octave = (double)scale[lev[0]] / (double)scale[lev[1]];
        if (ratio_dist * p->ratio_factor < ratio_octave || ratio_dist > ratio_octave * p->ratio_factor) continue;
        for (int c = 0; c < 3; ++c) xyz[3 * k + c] = (float)X[c];
        ok[k] = 1;
    }
}
