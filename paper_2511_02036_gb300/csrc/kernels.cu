// Kernels of the local-mapping search path for sm_103a.
//
//   ingest_kernel      Sec. IV-B  keyframe enters the store: group keypoints by BoW node key,
//                                 build the node-key bucket table and the 64x48 projection-grid
//                                 index (one CTA per keyframe)
//   search_kernel      Sec. IV-C  one CTA per (new KF, neighbour) pair: fundamental matrix ->
//                                 node join (bucket lookup) -> Hamming + epipolar gate ->
//                                 best/second -> accept -> one match per target -> rotation
//                                 histogram -> top-3 bins -> ordered compaction
//   fuse_kernel        Sec. IV-D  fusion search, one thread per map point: projection gates ->
//                                 grid window -> reprojection gate -> best Hamming
//   copy_kernel                   per-item counts -> offsets; regions -> one dense array
//   pair_* / fuse_*    plain form: one pair per launch sequence, global scratch
//
// Floating point: every gate is evaluated with explicit round-to-nearest intrinsics in the
// order stated next to it (no contraction, IEEE division and square root), so that a
// decision equals the one of a plain float32 evaluation of the same expression.
#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "tm.h"

namespace tmap {

// Bounds-checking build (-DTM_DEBUG_BOUNDS): every index that comes from data (bucket tables,
// grid lists, match lists, query lists) is checked against the array it indexes before use;
// the first failed check records its site here and the index is clamped into range, so that
// the run completes and the host reads the site (tm_debug_bounds).  In the normal build the
// check is the identity.
#ifdef TM_DEBUG_BOUNDS
__device__ unsigned int g_bounds_site;
#endif

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ int guard(int i, int n, unsigned site) {
#ifdef TM_DEBUG_BOUNDS
    if (i < 0 || i >= n) {
        atomicCAS(&g_bounds_site, 0u, site);
        return n > 0 ? (i < 0 ? 0 : n - 1) : 0;
    }
#else
    (void)n;
    (void)site;
#endif
    return i;
}

// ------------------------------------------------------------------------- arithmetic

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// Pyramid scale of a level: 1.2^l by repeated float multiplication.
__device__ __forceinline__ float level_scale(int l) {
    float s = 1.0f;
    for (int k = 0; k < l; ++k) s = fmul(s, 1.2f);
    return s;
}

// Fundamental matrix of the pair (Sec. IV-C epipolar validation): relative motion
// R = R_Q R_T^T, t = t_Q - R t_T; F = K^-T [t]x R K^-1 in float64, products evaluated
// ((K^-T [t]x) R) K^-1, each entry of each 3x3 product summed over k = 0, 1, 2 in that order,
// then rounded to float32.  x_Q^T F x_T = 0.
// Computed by nine lanes of a warp, lane e = 3r + c holding entry (r, c) of each 3x3 product,
// so that each lane runs ~25 float64 operations rather than one thread running ~240 (float64
// issue is narrow on this part).  All lanes of the warp call it; lanes 0..8 write F.
__device__ __noinline__ void fundamental_lanes(const CamConst &cam, const double *Tq, const double *Tt,
                                               float *Fout) {
    const int lane = (int)(threadIdx.x & 31u);
    const int e = lane < 9 ? lane : 0, r = e / 3, c = e % 3;
    // R = R_Q R_T^T
    double R = dmul(Tq[r * 4 + 0], Tt[c * 4 + 0]);
    R = dadd(R, dmul(Tq[r * 4 + 1], Tt[c * 4 + 1]));
    R = dadd(R, dmul(Tq[r * 4 + 2], Tt[c * 4 + 2]));
    // t = t_Q - R t_T (row r of R from lanes 3r .. 3r + 2)
    const double Rr0 = __shfl_sync(kFull, R, 3 * r), Rr1 = __shfl_sync(kFull, R, 3 * r + 1),
                 Rr2 = __shfl_sync(kFull, R, 3 * r + 2);
    double s = dmul(Rr0, Tt[0 * 4 + 3]);
    s = dadd(s, dmul(Rr1, Tt[1 * 4 + 3]));
    s = dadd(s, dmul(Rr2, Tt[2 * 4 + 3]));
    const double tr = dsub(Tq[r * 4 + 3], s);
    const double t0 = __shfl_sync(kFull, tr, 0), t1 = __shfl_sync(kFull, tr, 3), t2 = __shfl_sync(kFull, tr, 6);
    const double tx[9] = {0.0, -t2, t1, t2, 0.0, -t0, -t1, t0, 0.0};
    const double Kinv[9] = {cam.kinv[0], 0.0, cam.kinv[1], 0.0, cam.kinv[2], cam.kinv[3], 0.0, 0.0, 1.0};
    // A = K^-T [t]x
    double Am = dmul(Kinv[0 * 3 + r], tx[0 * 3 + c]);
    Am = dadd(Am, dmul(Kinv[1 * 3 + r], tx[1 * 3 + c]));
    Am = dadd(Am, dmul(Kinv[2 * 3 + r], tx[2 * 3 + c]));
    // B = A R
    const double Ar0 = __shfl_sync(kFull, Am, 3 * r), Ar1 = __shfl_sync(kFull, Am, 3 * r + 1),
                 Ar2 = __shfl_sync(kFull, Am, 3 * r + 2);
    const double R0c = __shfl_sync(kFull, R, c), R1c = __shfl_sync(kFull, R, 3 + c),
                 R2c = __shfl_sync(kFull, R, 6 + c);
    double B = dmul(Ar0, R0c);
    B = dadd(B, dmul(Ar1, R1c));
    B = dadd(B, dmul(Ar2, R2c));
    // F = B K^-1
    const double Br0 = __shfl_sync(kFull, B, 3 * r), Br1 = __shfl_sync(kFull, B, 3 * r + 1),
                 Br2 = __shfl_sync(kFull, B, 3 * r + 2);
    double F = dmul(Br0, Kinv[0 * 3 + c]);
    F = dadd(F, dmul(Br1, Kinv[1 * 3 + c]));
    F = dadd(F, dmul(Br2, Kinv[2 * 3 + c]));
    if (lane < 9) Fout[lane] = __double2float_rn(F);
}

// The same F for three pairs at once: lanes 9 k .. 9 k + 8 take pair k (k = 0, 1, 2; lanes
// 27 .. 31 repeat pair 2's first lanes and write nothing), each lane one entry, with the
// operation order of fundamental_lanes.  Tq[k], Tt[k]: the poses of pair k (null: no pair k,
// its lanes idle); lane 9 k + e writes Fout[k][e].
__device__ __noinline__ void fundamental_lanes3(const CamConst &cam, const double *const *Tq, const double *const *Tt,
                                                float (*Fout)[12]) {
    const int lane = (int)(threadIdx.x & 31u);
    const int k = lane < 27 ? lane / 9 : 2, e = lane < 27 ? lane % 9 : lane - 27, r = e / 3, c = e % 3;
    const int gb = 9 * k;  // the group's first lane
    const double *tq = Tq[k] ? Tq[k] : Tq[0], *tt = Tt[k] ? Tt[k] : Tt[0];
    double R = dmul(tq[r * 4 + 0], tt[c * 4 + 0]);
    R = dadd(R, dmul(tq[r * 4 + 1], tt[c * 4 + 1]));
    R = dadd(R, dmul(tq[r * 4 + 2], tt[c * 4 + 2]));
    const double Rr0 = __shfl_sync(kFull, R, gb + 3 * r), Rr1 = __shfl_sync(kFull, R, gb + 3 * r + 1),
                 Rr2 = __shfl_sync(kFull, R, gb + 3 * r + 2);
    double s = dmul(Rr0, tt[0 * 4 + 3]);
    s = dadd(s, dmul(Rr1, tt[1 * 4 + 3]));
    s = dadd(s, dmul(Rr2, tt[2 * 4 + 3]));
    const double tr = dsub(tq[r * 4 + 3], s);
    const double t0 = __shfl_sync(kFull, tr, gb + 0), t1 = __shfl_sync(kFull, tr, gb + 3),
                 t2 = __shfl_sync(kFull, tr, gb + 6);
    const double tx[9] = {0.0, -t2, t1, t2, 0.0, -t0, -t1, t0, 0.0};
    const double Kinv[9] = {cam.kinv[0], 0.0, cam.kinv[1], 0.0, cam.kinv[2], cam.kinv[3], 0.0, 0.0, 1.0};
    double Am = dmul(Kinv[0 * 3 + r], tx[0 * 3 + c]);
    Am = dadd(Am, dmul(Kinv[1 * 3 + r], tx[1 * 3 + c]));
    Am = dadd(Am, dmul(Kinv[2 * 3 + r], tx[2 * 3 + c]));
    const double Ar0 = __shfl_sync(kFull, Am, gb + 3 * r), Ar1 = __shfl_sync(kFull, Am, gb + 3 * r + 1),
                 Ar2 = __shfl_sync(kFull, Am, gb + 3 * r + 2);
    const double R0c = __shfl_sync(kFull, R, gb + c), R1c = __shfl_sync(kFull, R, gb + 3 + c),
                 R2c = __shfl_sync(kFull, R, gb + 6 + c);
    double B = dmul(Ar0, R0c);
    B = dadd(B, dmul(Ar1, R1c));
    B = dadd(B, dmul(Ar2, R2c));
    const double Br0 = __shfl_sync(kFull, B, gb + 3 * r), Br1 = __shfl_sync(kFull, B, gb + 3 * r + 1),
                 Br2 = __shfl_sync(kFull, B, gb + 3 * r + 2);
    double F = dmul(Br0, Kinv[0 * 3 + c]);
    F = dadd(F, dmul(Br1, Kinv[1 * 3 + c]));
    F = dadd(F, dmul(Br2, Kinv[2 * 3 + c]));
    if (lane < 27 && Tq[k]) Fout[k][e] = __double2float_rn(F);
}

// Epipolar line of a query in the target image: l = F^T x_Q = (a, b, c).
struct Line { float a, b, c; };
__device__ __forceinline__ Line epi_line(const float *F, float xq, float yq) {
    Line l;
    l.a = fadd(fadd(fmul(xq, F[0]), fmul(yq, F[3])), F[6]);
    l.b = fadd(fadd(fmul(xq, F[1]), fmul(yq, F[4])), F[7]);
    l.c = fadd(fadd(fmul(xq, F[2]), fmul(yq, F[5])), F[8]);
    return l;
}
// dist^2 = num^2 / (a^2 + b^2) < thr, division-free: num^2 < thr * den.
__device__ __forceinline__ float epi_den(const Line &l) { return fadd(fmul(l.a, l.a), fmul(l.b, l.b)); }
__device__ __forceinline__ bool epi_pass_den(const Line &l, float den, float xt, float yt, float thr) {
    const float num = fadd(fadd(fmul(l.a, xt), fmul(l.b, yt)), l.c);
    return den > 0.0f && fmul(num, num) < fmul(thr, den);
}
__device__ __forceinline__ bool epi_pass(const Line &l, float xt, float yt, float thr) {
    return epi_pass_den(l, epi_den(l), xt, yt, thr);
}

// The epipole in T (ORB-family rejection): Q's camera centre C_Q = -R_Q^T t_Q, C = R_T C_Q +
// t_T, e = (fx * (C_x / C_z) + cx, fy * (C_y / C_z) + cy), float64 with sums left to right,
// rounded to float32 (+-inf or NaN when C_z = 0, which then rejects nothing).  One thread.
__device__ void epipole_of(const CamConst &cam, const double *Tq, const double *Tt, float *e) {
    double cq[3], c[3];
    for (int k = 0; k < 3; ++k) {
        double s = dmul(Tq[0 * 4 + k], Tq[0 * 4 + 3]);
        s = dadd(s, dmul(Tq[1 * 4 + k], Tq[1 * 4 + 3]));
        s = dadd(s, dmul(Tq[2 * 4 + k], Tq[2 * 4 + 3]));
        cq[k] = -s;
    }
    for (int r = 0; r < 3; ++r) {
        double s = dmul(Tt[r * 4 + 0], cq[0]);
        s = dadd(s, dmul(Tt[r * 4 + 1], cq[1]));
        s = dadd(s, dmul(Tt[r * 4 + 2], cq[2]));
        c[r] = dadd(s, Tt[r * 4 + 3]);
    }
    e[0] = __double2float_rn(dadd(dmul(cam.fx, __ddiv_rn(c[0], c[2])), cam.cx));
    e[1] = __double2float_rn(dadd(dmul(cam.fy, __ddiv_rn(c[1], c[2])), cam.cy));
}
// ORB-family pair-baseline skip: with T's median scene depth known (> 0), the pair is not
// searched when |C_Q - C_T| / depth < min_ratio (camera centres C = -R^T t; float64, sums
// left to right).  One thread.
__device__ bool pair_skipped(const double *Tq, const double *Tt, float depth, float min_ratio) {
    if (!(min_ratio > 0.0f && depth > 0.0f)) return false;
    double c[2][3];
    const double *P[2] = {Tq, Tt};
    for (int v = 0; v < 2; ++v)
        for (int k = 0; k < 3; ++k) {
            double s = dmul(P[v][0 * 4 + k], P[v][0 * 4 + 3]);
            s = dadd(s, dmul(P[v][1 * 4 + k], P[v][1 * 4 + 3]));
            s = dadd(s, dmul(P[v][2 * 4 + k], P[v][2 * 4 + 3]));
            c[v][k] = -s;
        }
    const double dx = dsub(c[0][0], c[1][0]), dy = dsub(c[0][1], c[1][1]), dz = dsub(c[0][2], c[1][2]);
    const double base = __dsqrt_rn(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
    return __ddiv_rn(base, (double)depth) < (double)min_ratio;
}
// Squared distance to the epipole below the level's threshold: the candidate is dropped.
__device__ __forceinline__ bool near_epipole(const float *e, float xt, float yt, float thr) {
    const float dx = fsub(e[0], xt), dy = fsub(e[1], yt);
    return fadd(fmul(dx, dx), fmul(dy, dy)) < thr;
}

// Rotation bin: 30 bins of 12 degrees over angle_Q - angle_T wrapped into [0, 360).
__device__ __forceinline__ int rot_bin(float aq, float at, int mode) {
    float rot = fsub(aq, at);
    if (rot < 0.0f) rot = fadd(rot, 360.0f);
    // mode 1: the ORB-family binning, nearest integer of rot * (1/30) (halves away from zero)
    int bin = mode == 1 ? (int)roundf(fmul(rot, 1.0f / 30.0f)) : (int)floorf(__fdiv_rn(rot, 12.0f));
    if (bin >= kBins || bin < 0) bin = 0;  // (< 0 only for angles outside [0, 360))
    return bin;
}

__device__ __forceinline__ int hamming(const uint4 &a0, const uint4 &a1, const uint4 &b0,
                                       const uint4 &b1) {
    return __popc(a0.x ^ b0.x) + __popc(a0.y ^ b0.y) + __popc(a0.z ^ b0.z) +
           __popc(a0.w ^ b0.w) + __popc(a1.x ^ b1.x) + __popc(a1.y ^ b1.y) +
           __popc(a1.z ^ b1.z) + __popc(a1.w ^ b1.w);
}

__device__ __forceinline__ int grid_cell(float v, float inv, int n) {
    float f = floorf(fmul(v, inv));
    f = fminf(fmaxf(f, 0.0f), float(n - 1));
    return int(f);
}

template <typename P>
__device__ __forceinline__ int lower_bound_u32(P a, int n, uint32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
template <typename P>
__device__ __forceinline__ int upper_bound_u32(P a, int lo, int n, uint32_t key) {
    int hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Exclusive position of this thread's flag among the flags of the block (thread order),
// and the block total.  Every thread of the block must call it.
__device__ __forceinline__ uint32_t block_scan_flag(bool flag, uint32_t *wtot, uint32_t &total) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned ball = __ballot_sync(kFull, flag);
    const uint32_t pre = __popc(ball & ((1u << lane) - 1u));
    if (lane == 0) wtot[warp] = __popc(ball);
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < nw ? wtot[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, v, o);
            if ((int)lane >= o) v += y;
        }
        if (lane < nw) wtot[lane] = v;
    }
    __syncthreads();
    const uint32_t base = warp ? wtot[warp - 1] : 0u;
    total = wtot[nw - 1];
    __syncthreads();
    return base + pre;
}

// Exclusive prefix sum of one value per thread over the block (thread order), and the block
// total.  Every thread of the block must call it.
__device__ __forceinline__ uint32_t block_scan_add(uint32_t x, uint32_t *wtot, uint32_t &total) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t v = x;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, o);
        if ((int)lane >= o) v += y;
    }
    if (lane == 31) wtot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nw ? wtot[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, t, o);
            if ((int)lane >= o) t += y;
        }
        if (lane < nw) wtot[lane] = t;
    }
    __syncthreads();
    const uint32_t r = v - x + (warp ? wtot[warp - 1] : 0u);
    total = wtot[nw - 1];
    __syncthreads();
    return r;
}

// Top-3 rotation bins as a bit mask (ties to the lower bin, empty bins never taken,
// 2nd/3rd dropped when 10*count < count of the 1st).
__device__ uint32_t top3_mask(const uint32_t *hist) {
    int top[3] = {-1, -1, -1};
    for (int r = 0; r < 3; ++r) {
        int best = -1;
        for (int b = 0; b < kBins; ++b) {
            if (hist[b] == 0 || b == top[0] || b == top[1]) continue;
            if (best < 0 || hist[b] > hist[best]) best = b;
        }
        top[r] = best;
    }
    uint32_t mask = 0;
    if (top[0] >= 0) {
        const uint32_t mx = hist[top[0]];
        mask |= 1u << top[0];
        for (int r = 1; r < 3; ++r)
            if (top[r] >= 0 && !(10u * hist[top[r]] < mx)) mask |= 1u << top[r];
    }
    return mask;
}

// Packed per-query result: target (13 bits), distance (9 bits), rotation bin (5 bits).
__device__ __forceinline__ uint32_t pack_res(uint32_t t, uint32_t d, uint32_t bin) {
    return (t << 14) | (d << 5) | bin;
}

// ------------------------------------------------------------------------- ingest

constexpr int kSortE = 2;            // keys per thread-chunk of the block merge sort
constexpr int kIngestThreads = 1024;
constexpr int kCellSortMax = 64;     // largest bucket or cell sorted in place (insertion sort)

// Sorts N unique keys in shared memory (N a power of two >= kSortE): every chunk of kSortE
// keys is sorted in registers, then runs are merged pairwise (merge path: each chunk of the
// output finds its split point by binary search and merges kSortE keys).  a and b are two
// buffers of N keys; returns the one holding the result.  All threads of the block call it.
template <typename K>
__device__ K *block_merge_sort(K *a, K *b, int N) {
    const int chunks = N / kSortE;
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        K r[kSortE];
#pragma unroll
        for (int k = 0; k < kSortE; ++k) r[k] = a[c * kSortE + k];
#pragma unroll
        for (int pass = 0; pass < kSortE; ++pass)
#pragma unroll
            for (int k = pass & 1; k + 1 < kSortE; k += 2)
                if (r[k + 1] < r[k]) { const K t = r[k]; r[k] = r[k + 1]; r[k + 1] = t; }
#pragma unroll
        for (int k = 0; k < kSortE; ++k) a[c * kSortE + k] = r[k];
    }
    __syncthreads();
    K *src = a, *dst = b;
    for (int L = kSortE; L < N; L <<= 1) {
        for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
            const int o = c * kSortE;
            const int pb = o & ~(2 * L - 1), d = o - pb;
            const K *A = src + pb, *B = src + pb + L;
            int lo = d > L ? d - L : 0, hi = d < L ? d : L;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A[mid] < B[d - 1 - mid]) lo = mid + 1; else hi = mid;
            }
            int ia = lo, ib = d - lo;
#pragma unroll
            for (int k = 0; k < kSortE; ++k) {
                const bool take_a = ib >= L || (ia < L && A[ia] < B[ib]);
                dst[o + k] = take_a ? A[ia++] : B[ib++];
            }
        }
        __syncthreads();
        K *t = src; src = dst; dst = t;
    }
    return src;
}

// Stored node key: a bijection of the 32-bit BoW node id (multiplication by an odd constant,
// then xor of the high half into the low half), so that equal keys are equal nodes and the top
// bits spread any id range evenly over the buckets.
__device__ __forceinline__ uint32_t node_key(uint32_t node) {
    const uint32_t y = node * 0x9E3779B1u;
    return y ^ (y >> 16);
}

// Stable counting sort of n small keys key(i) < nb (i = 0 .. n-1) into out[0, n) (the items
// i in key order, i ascending within a key), with start[k] = first output of key k (k <= nb).
// counts: nb words of shared memory.  Returns the largest count; each bucket is then ordered
// by the caller's rule (insertion sort) when that count is small.  All threads call it.
template <typename KeyF>
__device__ uint32_t block_count_place(int n, int nb, KeyF key, uint32_t *counts, uint16_t *start,
                                      uint16_t *out, uint32_t *wtot, uint32_t *s_max) {
    const int tid = threadIdx.x, bs = blockDim.x;
    for (int k = tid; k < nb; k += bs) counts[k] = 0u;
    if (tid == 0) *s_max = 0u;
    __syncthreads();
    for (int i = tid; i < n; i += bs) atomicAdd(&counts[key(i)], 1u);
    __syncthreads();
    const int per = (nb + bs - 1) / bs, cb = min(tid * per, nb), ce = min(cb + per, nb);
    uint32_t sum = 0, mx = 0;
    for (int k = cb; k < ce; ++k) { sum += counts[k]; mx = max(mx, counts[k]); }
    uint32_t total;
    uint32_t run = block_scan_add(sum, wtot, total);
    for (int k = cb; k < ce; ++k) {
        const uint32_t c = counts[k];
        start[k] = (uint16_t)run;
        counts[k] = run;  // placement cursor
        run += c;
    }
    if (tid == 0) start[nb] = (uint16_t)n;
    mx = __reduce_max_sync(kFull, mx);
    if ((tid & 31) == 0) atomicMax(s_max, mx);
    __syncthreads();
    for (int i = tid; i < n; i += bs) out[atomicAdd(&counts[key(i)], 1u)] = (uint16_t)i;
    __syncthreads();
    return *s_max;
}

// Puts every segment [start[k], start[k+1]) of v in ascending order of less(.,.) (insertion
// sort, one thread per segment).  All threads call it.
template <typename Less>
__device__ void block_sort_segments(uint16_t *v, const uint16_t *start, int nb, Less less) {
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const int b = start[k], e = start[k + 1];
        for (int i = b + 1; i < e; ++i) {
            const uint16_t x = v[i];
            int j = i - 1;
            while (j >= b && less(x, v[j])) { v[j + 1] = v[j]; --j; }
            v[j + 1] = x;
        }
    }
    __syncthreads();
}

// Dynamic shared memory of the ingest kernel for a slot capacity (N = power of two >= cap):
// kbuf 16N bytes (the fallback merge sorts; otherwise node keys, cells, cell lists) and the
// node order 2N bytes.
__host__ __device__ constexpr size_t ingest_pow2(int cap) {
    size_t N = kSortE;
    while (N < (size_t)cap) N <<= 1;
    return N;
}

// One CTA per keyframe entering the store (Sec. IV-B).  Keypoints are put in node-key order
// (stable: caller order within a node) by a counting sort over the key's top 12 bits and an
// insertion sort inside each bucket; every keypoint array is gathered into that order while
// each keypoint's projection-grid cell is taken; the grid's cell lists come from a second
// counting sort (node order inside each cell).  A bucket or cell with more than kCellSortMax
// keypoints switches that sort to a merge sort of (key, position) pairs.  40 registers a
// thread: a 1024-thread CTA leaves a third of the register file to the prep CTAs beside it.
__global__ void __maxnreg__(40) ingest_kernel(IngestArgs A) {
    extern __shared__ __align__(16) unsigned char ism[];
    __shared__ uint32_t counts[kBuckets > kGridCells ? kBuckets : kGridCells];  // both sorts
    __shared__ uint16_t bstart[kBuckets + 1];
    __shared__ uint16_t gs[kGridCells + 1];
    __shared__ uint32_t wtot[32];
    __shared__ uint32_t s_max;
    const IngestJob &job = A.jobs[blockIdx.x];
    const int n = job.n;
    const int tid = threadIdx.x, bs = blockDim.x;
    int N = kSortE;
    while (N < n) N <<= 1;
    const int NC = (int)ingest_pow2(A.cap);  // carve by capacity (same offsets for every CTA)
    unsigned long long *k0 = reinterpret_cast<unsigned long long *>(ism);
    unsigned long long *k1 = k0 + N;
    uint32_t *skey = reinterpret_cast<uint32_t *>(ism + 8 * (size_t)NC);   // inside k1's region
    uint16_t *ord = reinterpret_cast<uint16_t *>(ism + 16 * (size_t)NC);
    const SlotLayout L = SlotLayout::make(A.cap);
    unsigned char *base = job.slot;
    // node keys in caller order
    for (int i = tid; i < n; i += bs) skey[i] = node_key(A.node[job.src + i]);
    __syncthreads();
    const uint32_t bmax = block_count_place(
        n, kBuckets, [&](int i) { return (int)(skey[i] >> (32 - kBucketBits)); }, counts, bstart, ord,
        wtot, &s_max);
    if (bmax <= (uint32_t)kCellSortMax) {
        block_sort_segments(ord, bstart, kBuckets, [&](uint16_t x, uint16_t y) {
            return skey[x] < skey[y] || (skey[x] == skey[y] && x < y);
        });
    } else {
        for (int i = tid; i < N; i += bs)
            k0[i] = i < n ? ((unsigned long long)skey[i] << 32) | (unsigned)i : ~0ull - (unsigned long long)i;
        __syncthreads();
        const unsigned long long *sorted = block_merge_sort(k0, k1, N);
        for (int p = tid; p < n; p += bs) ord[p] = (uint16_t)(sorted[p] & 0xFFFFu);
        __syncthreads();
    }
    // gather into node order; each keypoint's cell.  kbuf now holds: c0 [N] u32 | c1 [N] u32
    // (fallback grid sort), pcell [N] u16 and glist [N] u16 after them.
    uint32_t *c0 = reinterpret_cast<uint32_t *>(ism), *c1 = c0 + N;
    uint16_t *pcell = reinterpret_cast<uint16_t *>(ism + 8 * (size_t)NC);
    uint16_t *glist = pcell + NC;
    uint4 *desc = reinterpret_cast<uint4 *>(base + L.desc);
    float2 *xy = reinterpret_cast<float2 *>(base + L.xy);
    float *angle = reinterpret_cast<float *>(base + L.angle);
    uint32_t *node = reinterpret_cast<uint32_t *>(base + L.node);
    uint16_t *orig = reinterpret_cast<uint16_t *>(base + L.orig);
    uint16_t *pos = reinterpret_cast<uint16_t *>(base + L.pos);
    uint8_t *level = base + L.level;
    for (int p = tid; p < n; p += bs) {
        const uint32_t o = (uint32_t)guard(ord[p], n, 19);
        const uint32_t s = job.src + o;
        const uint4 d0 = A.desc[2 * s], d1 = A.desc[2 * s + 1];
        const float2 v = A.xy[s];
        const float an = A.angle[s];
        const uint32_t nd = A.node[s];
        const uint8_t lv = A.level[s];
        desc[2 * p] = d0;
        desc[2 * p + 1] = d1;
        xy[p] = v;
        angle[p] = an;
        node[p] = node_key(nd);
        orig[p] = (uint16_t)o;
        pos[o] = (uint16_t)p;
        level[p] = lv < kLevels ? lv : (uint8_t)(kLevels - 1);
        pcell[p] = (uint16_t)(grid_cell(v.y, A.cell_h_inv, kGridRows) * kGridCols +
                              grid_cell(v.x, A.cell_w_inv, kGridCols));
    }
    __syncthreads();
    const uint32_t cmax = block_count_place(
        n, kGridCells, [&](int p) { return (int)pcell[p]; }, counts, gs, glist, wtot, &s_max);
    uint16_t *gitems = reinterpret_cast<uint16_t *>(base + L.grid_items);
    if (cmax <= (uint32_t)kCellSortMax) {
        block_sort_segments(glist, gs, kGridCells, [](uint16_t x, uint16_t y) { return x < y; });
        for (int k = tid; k < n; k += bs) gitems[k] = glist[k];
    } else {
        for (int p = tid; p < N; p += bs)
            c0[p] = p < n ? ((uint32_t)pcell[p] << 16) | (uint32_t)p : 0xFFFFFFFFu - (uint32_t)p;
        __syncthreads();
        const uint32_t *ck = block_merge_sort(c0, c1, N);
        for (int k = tid; k < n; k += bs) gitems[k] = (uint16_t)(ck[k] & 0xFFFFu);
    }
    uint16_t *gstart = reinterpret_cast<uint16_t *>(base + L.grid_start);
    for (int c = tid; c <= kGridCells; c += bs) gstart[c] = gs[c];
    uint16_t *bst = reinterpret_cast<uint16_t *>(base + L.bstart);
    for (int b = tid; b <= kBuckets; b += bs) bst[b] = bstart[b];
    if (tid == 0) {
        KfHeader *h = reinterpret_cast<KfHeader *>(base);
        h->n = n;
        h->cap = A.cap;
        for (int k = 0; k < 12; ++k) h->Tcw[k] = job.Tcw[k];
    }
}

// Copies `bytes` from src to dst with the widest accesses both alignments allow; all threads
// of the CTA take part.
__device__ __forceinline__ void block_copy(unsigned char *dst, const unsigned char *src, size_t bytes) {
    const int tid = threadIdx.x, bs = blockDim.x;
    const uintptr_t al = reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes;
    if ((al & 15) == 0) {
        const uint4 *s = reinterpret_cast<const uint4 *>(src);
        uint4 *d = reinterpret_cast<uint4 *>(dst);
        for (size_t k = tid; k < bytes / 16; k += bs) d[k] = s[k];
    } else if ((al & 3) == 0) {
        const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
        uint32_t *d = reinterpret_cast<uint32_t *>(dst);
        for (size_t k = tid; k < bytes / 4; k += bs) d[k] = s[k];
    } else {
        for (size_t k = tid; k < bytes; k += bs) dst[k] = src[k];
    }
}

struct StageOffsets { size_t o[5]; };

// One CTA per keyframe in page-locked host memory: its five arrays into the staging area.
__global__ void __launch_bounds__(256) stage_gather_kernel(const GatherJob *jobs, unsigned char *base,
                                                           StageOffsets offs) {
    const GatherJob g = jobs[blockIdx.x];
    const uint32_t elt[5] = {32, 8, 4, 4, 1};  // desc, xy, angle, node, level
    for (int q = 0; q < 5; ++q)
        block_copy(base + offs.o[q] + (size_t)g.dst * elt[q], g.src[q], (size_t)g.n * elt[q]);
}

// ------------------------------------------------------------------------- TMA helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's (and, after a CTA barrier, the CTA's) generic-proxy shared-memory
// accesses before later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Hint: bring [p, p + bytes) into L2 (16-byte aligned address, size a multiple of 16; no
// completion to wait for).
__device__ __forceinline__ void bulk_prefetch_l2(const void *p, uint32_t bytes) {
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// The waiting thread is suspended until the phase completes or about 20 us pass (the time
// hint, ns), so that waiting warps do not take issue slots from the CTAs beside them.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete, at most `limit` SM clock cycles
// (~2 s by default).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Bounded wait for a CTA's bulk copies (phase 0 of bar).  With the `starve` test hook the
// copies are awaited as usual and then a second barrier that nothing arrives at is awaited, so
// that the bound runs out with no copy in flight.  Every thread of the CTA calls it; `never`
// is initialized (count 1) by the thread that initialized bar.
__device__ __forceinline__ bool staged_wait(uint64_t *bar, uint64_t *never, const BatchArgs &A) {
    bool ok = mbar_wait_bounded(bar, 0, A.wait_limit);
    if (ok && A.starve) ok = mbar_wait_bounded(never, 0, A.wait_limit);
    return ok;
}

// ------------------------------------------------------------------------- batch pipeline
//
// A batch runs as two branches of a graph, each ending with the compaction of its own records:
//   search   search_kernel, one CTA per pair (largest first): everything of Sec. IV-C for the
//            pair, with the neighbour's node index, the winners, the accepted matches and the
//            results in shared memory.  It reads a new keyframe from its staged arrays, so it
//            runs beside the ingest.  Then copy_kernel over the search items.
//   store    ingest_kernel, then fuse_kernel (CTA per 512 map points of a step: projection
//            gates, grid window in the staged target, best Hamming), then copy_kernel over the
//            fusion items (per-item counts -> offsets, per-item regions -> dense output,
//            comparison totals).

struct FuseK {
    float R[9], t[3], O[3], scale[kLevels], thr[kLevels];
};

// Adds a per-thread count to *dst: one atomic per warp.  All threads of the warp call.
__device__ __forceinline__ void warp_count(uint32_t v, uint32_t *dst) {
    const uint32_t sum = __reduce_add_sync(kFull, v);
    if ((threadIdx.x & 31u) == 0 && sum) atomicAdd(dst, sum);
}

// Top-3 rotation bins by one warp (same rule as top3_mask).  All lanes of the warp call.
__device__ __forceinline__ uint32_t top3_mask_warp(const uint32_t *hist) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t c = lane < (uint32_t)kBins ? hist[lane] : 0u;
    uint32_t taken = 0, mask = 0, mx = 0;
    for (int r = 0; r < 3; ++r) {
        // highest count wins, ties to the lowest bin; empty or taken bins never
        const uint32_t key = (c > 0 && !((taken >> lane) & 1u)) ? (c << 5) | (31u - lane) : 0u;
        const uint32_t m = __reduce_max_sync(kFull, key);
        if (m == 0) break;
        const uint32_t b = 31u - (m & 31u), cnt = m >> 5;
        if (r == 0) mx = cnt;
        if (r == 0 || !(10u * cnt < mx)) mask |= 1u << b;
        taken |= 1u << b;
    }
    return mask;
}

// A map point as the fusion reads it (Sec. IV-D's map-point data).
struct MapPoint {
    float X, Y, Z, nx, ny, nz, mind, maxd;
    uint4 d0, d1;
};
// Every global load of a map point, issued together.
__device__ __forceinline__ MapPoint load_mp(const float *pos, const float *normal, const uint4 *desc,
                                            float mind, float maxd) {
    MapPoint q;
    q.X = pos[0]; q.Y = pos[1]; q.Z = pos[2];
    q.nx = normal[0]; q.ny = normal[1]; q.nz = normal[2];
    q.d0 = desc[0]; q.d1 = desc[1];
    q.mind = mind; q.maxd = maxd;
    return q;
}

// Where a map point projects into the target (Sec. IV-D's gates before the window): pixel
// (u, v), window half-size r and pyramid level pl, and the grid cells of the window packed as
// cx0 | cx1 << 8 | cy0 << 16 | cy1 << 24.
struct FuseProj {
    float u, v, r;
    int pl;
    uint32_t cells;
};
// The projection gates of one map point: in front of the camera, inside the image, within its
// scale-invariance distance range, viewing angle below 60 degrees; then its predicted level
// and window.  False when a gate rejects it.
__device__ __forceinline__ bool fuse_project(const CamConst &cam, const FuseConst &fp, const FuseK &K,
                                             float X, float Y, float Z, float nx, float ny, float nz,
                                             float mind, float maxd, FuseProj &P) {
    const float xc = fadd(fadd(fadd(fmul(K.R[0], X), fmul(K.R[1], Y)), fmul(K.R[2], Z)), K.t[0]);
    const float yc = fadd(fadd(fadd(fmul(K.R[3], X), fmul(K.R[4], Y)), fmul(K.R[5], Z)), K.t[1]);
    const float zc = fadd(fadd(fadd(fmul(K.R[6], X), fmul(K.R[7], Y)), fmul(K.R[8], Z)), K.t[2]);
    if (!(zc > 0.0f)) return false;
    const float x = __fdiv_rn(xc, zc), y = __fdiv_rn(yc, zc);
    const float u = fadd(fmul(float(cam.fx), x), float(cam.cx));
    const float v = fadd(fmul(float(cam.fy), y), float(cam.cy));
    if (!(u >= 0.0f && u < float(cam.width) && v >= 0.0f && v < float(cam.height))) return false;
    const float pox = fsub(X, K.O[0]), poy = fsub(Y, K.O[1]), poz = fsub(Z, K.O[2]);
    const float dist = __fsqrt_rn(fadd(fadd(fmul(pox, pox), fmul(poy, poy)), fmul(poz, poz)));
    if (dist < mind || dist > maxd) return false;
    const float cosv = fadd(fadd(fmul(pox, nx), fmul(poy, ny)), fmul(poz, nz));
    if (cosv < fmul(0.5f, dist)) return false;
    int pl = kLevels - 1;
    for (int l = 0; l < kLevels; ++l)
        if (fmul(dist, K.scale[l]) >= maxd) { pl = l; break; }
    const float r = fmul(fp.radius_scale, K.scale[pl]);
    // cells of the window: a keypoint passing |x - u| < r in float32 lies within r + 1e-6 px of
    // u, so edges moved out by 0.01 px bound every such keypoint, and the cell of an edge bounds
    // the cell of the keypoint (rounding and floor are monotone)
    const int cx0 = grid_cell(fsub(fsub(u, r), 0.01f), cam.cell_w_inv, kGridCols);
    const int cx1 = grid_cell(fadd(fadd(u, r), 0.01f), cam.cell_w_inv, kGridCols);
    const int cy0 = grid_cell(fsub(fsub(v, r), 0.01f), cam.cell_h_inv, kGridRows);
    const int cy1 = grid_cell(fadd(fadd(v, r), 0.01f), cam.cell_h_inv, kGridRows);
    P.u = u;
    P.v = v;
    P.r = r;
    P.pl = pl;
    P.cells = (uint32_t)cx0 | (uint32_t)cx1 << 8 | (uint32_t)cy0 << 16 | (uint32_t)cy1 << 24;
    return true;
}

// The window search of a projected map point (descriptor m0 m1): every keypoint of the window's
// cells at level pl or pl - 1 within r of (u, v) on both axes and inside the reprojection
// gate is compared; returns the packed (distance << 16 | caller keypoint) of the best one
// under hamming_max, or kNone; adds the window comparisons to cmp.
__device__ __forceinline__ uint32_t fuse_window(const KfView &T, int nT, const FuseConst &fp, const FuseK &K,
                                                const FuseProj &P, const uint4 &m0, const uint4 &m1,
                                                uint32_t &cmp) {
    const float u = P.u, v = P.v, r = P.r;
    const int pl = P.pl;
    const int cx0 = (int)(P.cells & 0xFFu), cx1 = (int)((P.cells >> 8) & 0xFFu);
    const int cy0 = (int)((P.cells >> 16) & 0xFFu), cy1 = (int)(P.cells >> 24);
    uint32_t best = kNone;  // (dist << 16) | caller keypoint index
    for (int cy = cy0; cy <= cy1; ++cy) {
        const int c0 = cy * kGridCols + cx0, c1 = cy * kGridCols + cx1;
        const int k0 = T.grid_start[c0], k1 = guard(T.grid_start[c1 + 1], nT + 1, 11);
        for (int k = k0; k < k1; ++k) {
            const int j = guard(T.grid_items[k], nT, 12);
            const int lv = T.level[j];
            if (lv != pl && lv != pl - 1) continue;
            const float2 xt = T.xy[j];
            if (!(fabsf(fsub(xt.x, u)) < r && fabsf(fsub(xt.y, v)) < r)) continue;
            ++cmp;
            const float ex = fsub(u, xt.x), ey = fsub(v, xt.y);
            if (!(fadd(fmul(ex, ex), fmul(ey, ey)) <= K.thr[lv])) continue;
            const uint32_t d = (uint32_t)hamming(m0, m1, T.desc[2 * j], T.desc[2 * j + 1]);
            best = min(best, (d << 16) | (uint32_t)T.orig[j]);
        }
    }
    if (best == kNone || (int)(best >> 16) > fp.hamming_max) return kNone;
    return best;
}

// Fusion of one map point into keyframe T (Sec. IV-D): projection gates, then the window.
// Returns the packed (distance << 16 | keypoint) or kNone; adds window comparisons to cmp.
__device__ __forceinline__ uint32_t fuse_one(const KfView &T, int nT, const CamConst &cam,
                                             const FuseConst &fp, const FuseK &K,
                                             const MapPoint &q, uint32_t &cmp) {
    FuseProj P;
    if (!fuse_project(cam, fp, K, q.X, q.Y, q.Z, q.nx, q.ny, q.nz, q.mind, q.maxd, P)) return kNone;
    return fuse_window(T, nT, fp, K, P, q.d0, q.d1, cmp);
}

// Pose-derived constants of a fusion target: R, t in float32 and the camera centre
// O = -R^T t formed in float64 and rounded; scale and reprojection thresholds per level.
// Threads 0..39 of the calling CTA write K.
__device__ __forceinline__ void fuse_setup(const KfHeader *h, float chi2, FuseK &K) {
    const int tid = threadIdx.x;
    if (tid < 9) K.R[tid] = __double2float_rn(h->Tcw[(tid / 3) * 4 + tid % 3]);
    if (tid >= 16 && tid < 19) {
        const int c = tid - 16;
        K.t[c] = __double2float_rn(h->Tcw[c * 4 + 3]);
        double s = dmul(h->Tcw[0 * 4 + c], h->Tcw[0 * 4 + 3]);
        s = dadd(s, dmul(h->Tcw[1 * 4 + c], h->Tcw[1 * 4 + 3]));
        s = dadd(s, dmul(h->Tcw[2 * 4 + c], h->Tcw[2 * 4 + 3]));
        K.O[c] = __double2float_rn(-s);
    }
    if (tid >= 32 && tid < 32 + kLevels) {
        const float s = level_scale(tid - 32);
        K.scale[tid - 32] = s;
        K.thr[tid - 32] = fmul(chi2, fmul(s, s));
    }
}

// ---------------------------------------------------------------- search (S1-S6)

// Merge of two partial (best key, second distance) states of one query: the two smallest
// candidates of the union.  Associative and commutative; identity (kNone, 0xFFFF).
__device__ __forceinline__ void merge_best2(uint32_t &b, uint32_t &s, uint32_t ob, uint32_t os) {
    s = min(min(s, os), max(b, ob) >> 16);
    b = min(b, ob);
}

// Shared memory of the candidate rounds, by 32-bit shared address: explicit ld/st/atom.shared,
// so that every access of the hot loops is a shared-memory instruction with a 32-bit address.
__device__ __forceinline__ uint32_t ld_s32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ld_s16(uint32_t a) {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 ld_s128(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void st_s32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_s128(uint32_t a, const float4 &v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint32_t atom_s_min(uint32_t a, uint32_t v) {
    uint32_t o;
    asm volatile("atom.shared.min.u32 %0, [%1], %2;" : "=r"(o) : "r"(a), "r"(v) : "memory");
    return o;
}
__device__ __forceinline__ void red_s_min(uint32_t a, uint32_t v) {
    asm volatile("red.shared.min.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// The load only where p holds (no branch around it); v unchanged elsewhere.
__device__ __forceinline__ uint32_t ld_s32_if(bool p, uint32_t a, uint32_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.shared.u32 %0, [%1];\n\t}"
                 : "+r"(v)
                 : "r"(a), "r"((int)p));
    return v;
}
__device__ __forceinline__ uint2 ld_s64(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

// Read-only global loads through the non-coherent path.
template <typename V>
__device__ __forceinline__ V ldg(const V *p) { return __ldg(p); }

// A warp searches 32 Q queries at a time (a group, Q = 1 or 2 queries per lane): lane l
// takes positions 32 Q g + l (its query 0) and, with Q = 2, 32 Q g + 32 + l (its query 1).
//
// The loads of a warp's group that depend on nothing else: issued one group ahead, so that
// their latency overlaps the previous group's search.
template <int Q>
struct QLoad {
    uint32_t nk[Q];  // node keys or raw node ids
    uint32_t io[Q];  // caller indices
    int el[Q];       // eligible (1/0), or -1: not loaded yet (stored query keyframe with masks)
};
template <int Q>
__device__ __forceinline__ QLoad<Q> load_group(const BatchArgs &A, const WorkItem &w, int g) {
    const int lane = (int)(threadIdx.x & 31u);
    QLoad<Q> q;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const int p0 = g * 32 * Q + 32 * h;
        const bool in = lane < (int)w.nq - p0;
        const int p = in ? p0 + lane : 0;
        q.nk[h] = ldg(w.qnode + p);
        if (w.qorig) {
            q.io[h] = ldg(w.qorig + p);
            q.el[h] = !in ? 0 : (w.a == kNone ? 1 : -1);
        } else {
            q.io[h] = (uint32_t)p;
            q.el[h] = in && (w.a == kNone || ldg(A.masks + w.a + (uint32_t)p));
        }
    }
    return q;
}

// Shared addresses of the search CTA's arrays and of the calling warp's query tables.
struct SearchSmem {
    uint32_t tkey, bst, words, epos, win, pc, thr, thre;
    uint32_t rec;  // the warp's query records: second distance << 16 | first eligible entry
    uint32_t sb;   // the warp's best keys (distance << 16 | target position)
};
constexpr uint32_t kSecTimeout = 0xFFFEu;  // second-distance field: the query's dense tile timed out

// Eligible positions before position j (0 <= j <= nT): the count before j's word plus the
// eligible bits of the word below j.
__device__ __forceinline__ int eligible_before(const SearchSmem &M, int j) {
    const uint2 wd = ld_s64(M.words + 8 * (j >> 5));
    return (int)wd.y + __popc(wd.x & ((1u << (j & 31)) - 1u));
}

// One group (32 Q queries) of the CTA's pair, by one warp (Sec. IV-C).  Each lane finds its
// queries' candidates: the bucket of the node key, the run of equal keys inside it (keys
// ascend within a bucket; one pass over the lane's buckets counting the keys below and up to
// each key), the run's eligible targets (counts from the eligibility bitmap).  The (query,
// candidate) entries of the group are numbered by a warp prefix sum (a lane's query 0 entries,
// then its query 1 entries) and taken 32 per round, lane k handling entry k (its lane found by
// a binary search over the prefix sums), so that the warp waits ~ceil(entries / 32) rounds of
// candidate loads for the group.  An entry's lane folds its (distance << 16 | target) key
// into the query's state with two shared atomicMin: the first returns the previous best, and
// the larger of the two is a loser whose distance bounds the second (entries of one query in
// one round are serialized by the hardware; the result does not depend on their order).  A
// query whose best passes the distance and ratio tests gets its rotation bin, is listed in the
// pair's accepted list (global, `acc`) and claims its target (shared atomicMin of
// (distance << 16 | caller)).  kEpi, kEprej, kDense: the epipolar gate, the epipole
// rejection and dense node blocks are on (fixed per launch).
// wing: the pair's per-target winners in global memory when the pair is split over two CTAs
// (else null: in shared memory); the accepted queries are listed from acc[c + abase].
// The lookups of a group (the first part of search_group): per query of the lane, the count n
// of its eligible candidates and its first eligible entry elo; a dense-block query's (best key,
// second) from the tensor cores in b0 / s0 (its n then 0; else kNone / 0xFFFF).
template <int Q, bool kDense>
__device__ __forceinline__ void group_lookup(const BatchArgs &A, const WorkItem &w, const SearchSmem &M, int g,
                                             const QLoad<Q> &q, uint32_t &cmp, int (&c)[Q], int (&elo_out)[Q],
                                             uint32_t (&b0_out)[Q], uint32_t (&s0_out)[Q]) {
    const int lane = (int)(threadIdx.x & 31u);
    const int nT = (int)w.nt;
    uint32_t key[Q];
    int lo[Q], be[Q];
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        key[h] = w.qraw ? node_key(q.nk[h]) : q.nk[h];
        const uint32_t b = key[h] >> (32 - kBucketBits);
        lo[h] = guard((int)ld_s16(M.bst + 2 * b), nT + 1, 1);
        be[h] = guard((int)ld_s16(M.bst + 2 * b + 2), nT + 1, 2);
    }
    // one pass over the lane's buckets: keys below each query's key, and up to it
    int nlt[Q], nle[Q], len = 0;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        nlt[h] = nle[h] = 0;
        len = max(len, be[h] - lo[h]);
    }
    for (int t = 0; t < len; ++t) {
        bool pt[Q];
        uint32_t kt[Q];
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            pt[h] = lo[h] + t < be[h];
            kt[h] = ld_s32_if(pt[h], M.tkey + 4 * (lo[h] + t), 0u);
        }
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            nlt[h] += pt[h] && kt[h] < key[h];
            nle[h] += pt[h] && kt[h] <= key[h];
        }
    }
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const bool el = q.el[h] >= 0 ? q.el[h] != 0 : (ldg(A.masks + w.a + q.io[h]) != 0);
        const int elo = eligible_before(M, lo[h] + nlt[h]);
        int n = el ? eligible_before(M, lo[h] + nle[h]) - elo : 0;
        uint32_t b0 = kNone, s0 = 0xFFFFu;
        // a query of a dense node block: its candidates were compared on the tensor cores
        if (kDense && el && nle[h] - nlt[h] >= A.sp.dense_min) {
            cmp += (uint32_t)n;
            n = 0;
            const uint2 v = A.dres[w.c + (uint32_t)(g * 32 * Q + 32 * h + lane)];
            b0 = v.x;
            s0 = v.y == kNone ? kSecTimeout : v.y;
        }
        c[h] = n;
        elo_out[h] = elo;
        b0_out[h] = b0;
        s0_out[h] = s0;
    }
}

template <int Q, bool kDense>
__device__ __forceinline__ void group_results(const BatchArgs &A, const WorkItem &w, const KfView &T,
                                              const SearchSmem &M, uint32_t *nacc, int g, const QLoad<Q> &q,
                                              uint32_t &dfail, uint32_t *wing, uint32_t abase);

template <int Q, bool kEpi, bool kEprej, bool kDense>
__device__ __forceinline__ void search_group(const BatchArgs &A, const WorkItem &w, const KfView &T,
                                             const SearchSmem &M, uint32_t *nacc, int g, const QLoad<Q> &q,
                                             uint32_t &cmp, uint32_t &dfail, uint32_t *wing, uint32_t abase) {
    const int lane = (int)(threadIdx.x & 31u);
    const int nT = (int)w.nt, nQ = (int)w.nq;
    int c[Q], elo[Q];
    uint32_t b0[Q], s0[Q];
    group_lookup<Q, kDense>(A, w, M, g, q, cmp, c, elo, b0, s0);
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        st_s32(M.sb + 4 * (32 * h + lane), b0[h]);
        st_s32(M.rec + 4 * (32 * h + lane), (s0[h] << 16) | (uint32_t)elo[h]);
    }
    const int c0 = c[0], cl = Q > 1 ? c[0] + c[Q - 1] : c[0];
    int off = cl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, off, o);
        if (lane >= o) off += y;
    }
    const int total = __shfl_sync(kFull, off, 31);
    off -= cl;  // exclusive
    __syncwarp();
    for (int k0 = 0; k0 < total; k0 += 32) {
        const int k = k0 + lane;
        // owner lane: the last lane whose first entry is <= k (it has entries, as k < total)
        int o = 0;
#pragma unroll
        for (int s2 = 16; s2 >= 1; s2 >>= 1) {
            const int oo = __shfl_sync(kFull, off, o + s2);
            if (oo <= k) o += s2;
        }
        const int r = k - __shfl_sync(kFull, off, o);
        const int c0o = Q > 1 ? __shfl_sync(kFull, c0, o) : 0x7FFFFFFF;
        if (k < total) {
            const int h = r >= c0o ? 1 : 0;
            const int qi = o + 32 * h;  // state index of the entry's query
            const uint32_t rw = ld_s32(M.rec + 4 * qi), elo = rw & 0xFFFFu;
            const int j0 = guard((int)ld_s16(M.epos + 2 * guard((int)elo + r - (h ? c0o : 0), nT, 3)), nT, 4);
            const int pq = guard(g * 32 * Q + qi, nQ, 5);
            const uint4 a0 = ldg(w.qdesc + 2 * pq), a1 = ldg(w.qdesc + 2 * pq + 1);
            const uint4 t0 = ldg(T.desc + 2 * j0), t1 = ldg(T.desc + 2 * j0 + 1);
            const float2 xt = ldg(T.xy + j0);
            const uint32_t lv = ldg(T.level + j0);
            ++cmp;
            const uint32_t d = (uint32_t)hamming(a0, a1, t0, t1);
            // an entry farther than the query's second (as read at the round's start: the
            // second only decreases) changes neither its best nor its second: no gates needed
            bool pass = d <= (rw >> 16);
            if (kEpi && pass) {
                // l = F^T x_Q: a = (x F00 + y F10) + F20, b = (x F01 + y F11) + F21,
                // c = (x F02 + y F12) + F22; num = (a x_T + b y_T) + c, den = a^2 + b^2;
                // pass iff den > 0 and num^2 < thr den
                const float2 xq = ldg(w.qxy + pq);
                const float4 F0 = ld_s128(M.pc), F1 = ld_s128(M.pc + 16), F2 = ld_s128(M.pc + 32);
                const float la = fadd(fadd(fmul(xq.x, F0.x), fmul(xq.y, F0.w)), F1.z);
                const float lb = fadd(fadd(fmul(xq.x, F0.y), fmul(xq.y, F1.x)), F1.w);
                const float lc = fadd(fadd(fmul(xq.x, F0.z), fmul(xq.y, F1.y)), F2.x);
                const float num = fadd(fadd(fmul(la, xt.x), fmul(lb, xt.y)), lc);
                const float den = fadd(fmul(la, la), fmul(lb, lb));
                pass = den > 0.0f && fmul(num, num) < fmul(__uint_as_float(ld_s32(M.thr + 4 * lv)), den);
            }
            if (kEprej && pass) {
                const float ex = __uint_as_float(ld_s32(M.pc + 36)), ey = __uint_as_float(ld_s32(M.pc + 40));
                const float dx = fsub(ex, xt.x), dy = fsub(ey, xt.y);
                if (fadd(fmul(dx, dx), fmul(dy, dy)) < __uint_as_float(ld_s32(M.thre + 4 * lv))) pass = false;
            }
            if (pass) {
                const uint32_t bk = (d << 16) | (uint32_t)j0;
                const uint32_t old = atom_s_min(M.sb + 4 * qi, bk);
                // the record: second << 16 | first eligible entry, the entry fixed for the
                // query, so the minimum of the word is that of the second
                red_s_min(M.rec + 4 * qi, ((max(old, bk) >> 16) << 16) | elo);
            }
        }
    }
    __syncwarp();
    group_results<Q, kDense>(A, w, T, M, nacc, g, q, dfail, wing, abase);
}

// The results of a group (the last part of search_group), from its queries' states in M.sb /
// M.rec: a query whose best passes the distance and ratio tests gets its rotation bin, is listed
// in the pair's accepted list and claims its target.
template <int Q, bool kDense>
__device__ __forceinline__ void group_results(const BatchArgs &A, const WorkItem &w, const KfView &T,
                                              const SearchSmem &M, uint32_t *nacc, int g, const QLoad<Q> &q,
                                              uint32_t &dfail, uint32_t *wing, uint32_t abase) {
    const int lane = (int)(threadIdx.x & 31u);
    const int nT = (int)w.nt, nQ = (int)w.nq;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const int p = g * 32 * Q + 32 * h + lane;
        bool ok = false;
        uint32_t best = 0, j = 0;
        if (p < nQ) {
            const uint32_t bk = ld_s32(M.sb + 4 * (32 * h + lane)), sc = ld_s32(M.rec + 4 * (32 * h + lane)) >> 16;
            if (kDense && sc == kSecTimeout) dfail = 1u;  // the dense tile of this query timed out
            if (bk != kNone) {
                best = bk >> 16;
                ok = (int)best <= A.sp.hamming_max;
                if (ok && A.sp.ratio_num != 0 && sc != 0xFFFFu)
                    ok = (long long)A.sp.ratio_den * best < (long long)A.sp.ratio_num * sc;
                j = (uint32_t)guard((int)(bk & 0xFFFFu), nT, 6);
            }
        }
        const unsigned m = __ballot_sync(kFull, ok);
        if (m) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(nacc, (uint32_t)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (ok) {
                const uint32_t io = q.io[h];
                const uint32_t bin = A.sp.rot_filter ? (uint32_t)rot_bin(ldg(w.qangle + p), ldg(T.angle + j), A.sp.rot_mode) : 0u;
                const uint32_t e = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
                A.acc[w.c + (uint32_t)guard((int)(abase + e), nQ, 7)] =
                    make_uint2(io | (j << 16), (uint32_t)ldg(T.orig + j) | (best << 16) | (bin << 25));
                if (A.sp.resolve) {
                    if (wing) atomicMin(wing + j, (best << 16) | io);
                    else red_s_min(M.win + 4 * j, (best << 16) | io);
                }
            }
        }
    }
    __syncwarp();
}

// Entry form, join pass (Sec. IV-C candidate generation without the comparisons): the group's
// lookups as in search_group; each query's state (best key, second) starts in dres at kNone /
// 0xFFFF, and its candidates are appended to the batch's entry list (a warp prefix of the
// lanes' counts, one atomicAdd a warp).  An entry past ent_cap is not written and flags the
// pair (ovf), whose finalize then searches it in rounds.
template <int Q>
__device__ __forceinline__ void join_group(const BatchArgs &A, const WorkItem &w, const SearchSmem &M, int g,
                                           const QLoad<Q> &q, uint32_t &cmp, uint32_t slot, bool &ovf) {
    const int lane = (int)(threadIdx.x & 31u);
    const int nQ = (int)w.nq, nT = (int)w.nt;
    int c[Q], elo[Q];
    uint32_t b0[Q], s0[Q];
    group_lookup<Q, false>(A, w, M, g, q, cmp, c, elo, b0, s0);
    int cl = 0;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const int p = g * 32 * Q + 32 * h + lane;
        if (p < nQ) A.dres[w.c + (uint32_t)p] = make_uint2(kNone, 0xFFFFu);
        cl += c[h];
    }
    int off = cl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, off, o);
        if (lane >= o) off += y;
    }
    const uint32_t total = (uint32_t)__shfl_sync(kFull, off, 31);
    off -= cl;
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(A.nents, total);
    base = __shfl_sync(kFull, base, 0);
    cmp += (uint32_t)cl;
    if ((uint64_t)base + total > A.ent_cap) ovf = true;
    uint32_t e = base + (uint32_t)off;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const uint32_t p = (uint32_t)(g * 32 * Q + 32 * h + lane);
        for (int r = 0; r < c[h]; ++r, ++e) {
            const uint32_t j = (uint32_t)guard((int)ld_s16(M.epos + 2 * guard(elo[h] + r, nT, 33)), nT, 34);
            if (e < A.ent_cap) A.ents[e] = make_uint2(slot, (p << 16) | j);
        }
    }
}

// Entry form, finalize pass: the group's states as the entries left them, then its results as
// in search_group.
template <int Q>
__device__ __forceinline__ void final_group(const BatchArgs &A, const WorkItem &w, const KfView &T,
                                            const SearchSmem &M, uint32_t *nacc, int g, const QLoad<Q> &q,
                                            uint32_t &dfail, uint32_t *wing, uint32_t abase) {
    const int lane = (int)(threadIdx.x & 31u);
    const int nQ = (int)w.nq;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const int p = g * 32 * Q + 32 * h + lane;
        const uint2 v = p < nQ ? A.dres[w.c + (uint32_t)p] : make_uint2(kNone, 0xFFFFu);
        st_s32(M.sb + 4 * (32 * h + lane), v.x);
        st_s32(M.rec + 4 * (32 * h + lane), v.y << 16);
    }
    __syncwarp();
    group_results<Q, false>(A, w, T, M, nacc, g, q, dfail, wing, abase);
}

// Entry form, evaluation pass: one thread per (query, candidate) entry of the batch (a grid
// stride over the list): Hamming distance, epipolar gate (the same float32 operations as the
// rounds), and the query's state folded with two atomicMin as the rounds do in shared memory
// (the first returns the previous best; the larger of the two bounds the second), so that the
// states do not depend on the order in which the entries run.
constexpr int kEvalThreads = 256;
template <bool kEpi>
__global__ void __launch_bounds__(kEvalThreads) eval_kernel(BatchArgs A) {
    __shared__ float thr[kLevels];
    if (threadIdx.x < kLevels) {
        const float sc = level_scale((int)threadIdx.x);
        thr[threadIdx.x] = fmul(A.sp.epi_chi2, fmul(sc, sc));
    }
    __syncthreads();
    const uint32_t n = min(*A.nents, A.ent_cap);
    for (uint32_t e = blockIdx.x * kEvalThreads + threadIdx.x; e < n; e += gridDim.x * kEvalThreads) {
        const uint2 en = A.ents[e];
        const WorkItem *wp = A.sitems + guard((int)en.x, (int)A.n_units, 30);
        const uint32_t nq = wp->nq, nt = wp->nt, c = wp->c;
        const KfView T = KfView::at(wp->t, A.L);
        const int p = guard((int)(en.y >> 16), (int)nq, 31), j = guard((int)(en.y & 0xFFFFu), (int)nt, 32);
        const uint4 *qd = wp->qdesc;
        const uint4 a0 = ldg(qd + 2 * p), a1 = ldg(qd + 2 * p + 1);
        const uint4 t0 = ldg(T.desc + 2 * j), t1 = ldg(T.desc + 2 * j + 1);
        const float2 xt = ldg(T.xy + j);
        const uint32_t lv = ldg(T.level + j);
        const uint32_t d = (uint32_t)hamming(a0, a1, t0, t1);
        uint32_t *st = reinterpret_cast<uint32_t *>(A.dres + c + (uint32_t)p);
        // an entry farther than the query's second (read from L2; the second only decreases, so
        // a stale read only costs work) changes neither its best nor its second: no gates and no
        // atomics
        if (d > __ldcg(st + 1)) continue;
        bool pass = true;
        if (kEpi) {
            // l = F^T x_Q as in the rounds: a = (x F00 + y F10) + F20, b = (x F01 + y F11) + F21,
            // c = (x F02 + y F12) + F22; num = (a x_T + b y_T) + c, den = a^2 + b^2;
            // pass iff den > 0 and num^2 < thr den
            const float2 xq = ldg(wp->qxy + p);
            const float4 *pc = reinterpret_cast<const float4 *>(A.pconst + (size_t)kPairConst * wp->idx);
            const float4 F0 = ldg(pc), F1 = ldg(pc + 1), F2 = ldg(pc + 2);
            const float la = fadd(fadd(fmul(xq.x, F0.x), fmul(xq.y, F0.w)), F1.z);
            const float lb = fadd(fadd(fmul(xq.x, F0.y), fmul(xq.y, F1.x)), F1.w);
            const float lc = fadd(fadd(fmul(xq.x, F0.z), fmul(xq.y, F1.y)), F2.x);
            const float num = fadd(fadd(fmul(la, xt.x), fmul(lb, xt.y)), lc);
            const float den = fadd(fmul(la, la), fmul(lb, lb));
            pass = den > 0.0f && fmul(num, num) < fmul(thr[guard((int)lv, kLevels, 35)], den);
        }
        if (pass) {
            const uint32_t bk = (d << 16) | (uint32_t)j;
            const uint32_t old = atomicMin(st, bk);
            atomicMin(st + 1, max(old, bk) >> 16);
        }
    }
}

// The same group (64 queries, two per lane) in the per-lane form: after the same bucket
// lookups, each lane walks its own queries' candidates itself, in eligible-list order (both
// queries' candidates interleaved, for two independent load chains), keeping each query's
// (best key, second distance) in registers -- no prefix sums, no owner search, no shared
// atomics, at the price of lanes that idle while the lane with most candidates finishes.
// The state of a query is the same minimum over its candidates as in the rounds.  Default
// gates only (epipolar gate on or off, no epipole rejection, no dense blocks).
template <bool kEpi>
__device__ __forceinline__ void search_group_lane(const BatchArgs &A, const WorkItem &w, const KfView &T,
                                                  const SearchSmem &M, uint32_t *nacc, int g, const QLoad<2> &q,
                                                  uint32_t &cmp, uint32_t *wing, uint32_t abase) {
    constexpr int Q = 2;
    const int lane = (int)(threadIdx.x & 31u);
    const int nT = (int)w.nt, nQ = (int)w.nq;
    uint32_t key[Q];
    int lo[Q], be[Q];
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        key[h] = w.qraw ? node_key(q.nk[h]) : q.nk[h];
        const uint32_t b = key[h] >> (32 - kBucketBits);
        lo[h] = guard((int)ld_s16(M.bst + 2 * b), nT + 1, 1);
        be[h] = guard((int)ld_s16(M.bst + 2 * b + 2), nT + 1, 2);
    }
    int nlt[Q], nle[Q], len = 0;
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        nlt[h] = nle[h] = 0;
        len = max(len, be[h] - lo[h]);
    }
    for (int t = 0; t < len; ++t) {
        bool pt[Q];
        uint32_t kt[Q];
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            pt[h] = lo[h] + t < be[h];
            kt[h] = ld_s32_if(pt[h], M.tkey + 4 * (lo[h] + t), 0u);
        }
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            nlt[h] += pt[h] && kt[h] < key[h];
            nle[h] += pt[h] && kt[h] <= key[h];
        }
    }
    int c[Q], elo[Q];
    uint32_t bk[Q], sc[Q];
    float la[Q], lb[Q], lc[Q];
    uint4 a0[Q], a1[Q];
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const bool el = q.el[h] >= 0 ? q.el[h] != 0 : (ldg(A.masks + w.a + q.io[h]) != 0);
        elo[h] = eligible_before(M, lo[h] + nlt[h]);
        c[h] = el ? eligible_before(M, lo[h] + nle[h]) - elo[h] : 0;
        bk[h] = kNone;
        sc[h] = 0xFFFFu;
        la[h] = lb[h] = lc[h] = 0.0f;
        a0[h] = a1[h] = make_uint4(0u, 0u, 0u, 0u);
        if (c[h] > 0) {
            const int pq = guard(g * 32 * Q + 32 * h + lane, nQ, 5);
            a0[h] = ldg(w.qdesc + 2 * pq);
            a1[h] = ldg(w.qdesc + 2 * pq + 1);
            if (kEpi) {
                // l = F^T x_Q, the same expression as in the rounds
                const float2 xq = ldg(w.qxy + pq);
                const float4 F0 = ld_s128(M.pc), F1 = ld_s128(M.pc + 16), F2 = ld_s128(M.pc + 32);
                la[h] = fadd(fadd(fmul(xq.x, F0.x), fmul(xq.y, F0.w)), F1.z);
                lb[h] = fadd(fadd(fmul(xq.x, F0.y), fmul(xq.y, F1.x)), F1.w);
                lc[h] = fadd(fadd(fmul(xq.x, F0.z), fmul(xq.y, F1.y)), F2.x);
            }
        }
    }
    const int cm = max(c[0], c[1]);
    for (int t = 0; t < cm; ++t) {
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            if (t < c[h]) {
                const int j0 = guard((int)ld_s16(M.epos + 2 * guard(elo[h] + t, nT, 3)), nT, 4);
                const uint4 t0 = ldg(T.desc + 2 * j0), t1 = ldg(T.desc + 2 * j0 + 1);
                const float2 xt = ldg(T.xy + j0);
                const uint32_t lv = ldg(T.level + j0);
                ++cmp;
                const uint32_t d = (uint32_t)hamming(a0[h], a1[h], t0, t1);
                // an entry farther than the query's second changes neither its best nor second
                bool pass = d <= sc[h];
                if (kEpi && pass) {
                    const float num = fadd(fadd(fmul(la[h], xt.x), fmul(lb[h], xt.y)), lc[h]);
                    const float den = fadd(fmul(la[h], la[h]), fmul(lb[h], lb[h]));
                    pass = den > 0.0f && fmul(num, num) < fmul(__uint_as_float(ld_s32(M.thr + 4 * lv)), den);
                }
                if (pass) {
                    const uint32_t kk = (d << 16) | (uint32_t)j0;
                    sc[h] = min(sc[h], max(bk[h], kk) >> 16);
                    bk[h] = min(bk[h], kk);
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < Q; ++h) {
        const int p = g * 32 * Q + 32 * h + lane;
        bool ok = false;
        uint32_t best = 0, j = 0;
        if (p < nQ && bk[h] != kNone) {
            best = bk[h] >> 16;
            ok = (int)best <= A.sp.hamming_max;
            if (ok && A.sp.ratio_num != 0 && sc[h] != 0xFFFFu)
                ok = (long long)A.sp.ratio_den * best < (long long)A.sp.ratio_num * sc[h];
            j = (uint32_t)guard((int)(bk[h] & 0xFFFFu), nT, 6);
        }
        const unsigned m = __ballot_sync(kFull, ok);
        if (m) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(nacc, (uint32_t)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (ok) {
                const uint32_t io = q.io[h];
                const uint32_t bin = A.sp.rot_filter ? (uint32_t)rot_bin(ldg(w.qangle + p), ldg(T.angle + j), A.sp.rot_mode) : 0u;
                const uint32_t e = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
                A.acc[w.c + (uint32_t)guard((int)(abase + e), nQ, 7)] =
                    make_uint2(io | (j << 16), (uint32_t)ldg(T.orig + j) | (best << 16) | (bin << 25));
                if (A.sp.resolve) {
                    if (wing) atomicMin(wing + j, (best << 16) | io);
                    else red_s_min(M.win + 4 * j, (best << 16) | io);
                }
            }
        }
    }
}


// ---------------------------------------------------------------- dense node blocks (S3b)
//
// A query whose BoW node holds at least dense_min keypoints of the neighbour belongs to a
// dense block: all eligible queries of that node against all keypoints of the node in the
// neighbour (Sec. IV-C's candidate set, unchanged).  Their Hamming distances come from the
// tensor cores.  A descriptor bit b becomes the fp8 (e4m3) value +1 (b = 0) or -1 (b = 1), so
// the dot product of two descriptors is 256 - 2 * Hamming: an integer of magnitude <= 256,
// exact in the float32 accumulator whatever the summation order.
//
// dense_kernel: CTA (pair, split) takes every splits-th dense run of the neighbour (found in
// its node keys staged in shared memory).  Per run, tiles of 128 queries x 128 keypoints: both
// operands expanded into shared memory (K-major core matrices, no swizzle; two threads per
// row, one uint4 of the descriptor each), eight tcgen05.mma of K = 32 issued by one thread
// into a 128-lane x 128-column float32 accumulator in tensor memory, completion by
// tcgen05.commit on an mbarrier (bounded wait).  Then the two warps of each 32-lane group read
// their half of the columns of their lanes' rows (tcgen05.ld) and apply the epipolar gate and
// the (best, second) merge of the candidate rounds to each column; the halves are merged.  The
// query's state goes to dres; search_kernel counts the query's comparisons and takes that
// state instead of visiting its candidates.

constexpr int kDenseRows = 128;                    // M: queries per tile (accumulator lanes)
constexpr int kDenseCols = 128;                    // N per tile = tensor-memory columns
constexpr int kDenseThreads = 256;                 // two warps per 32-lane group: column halves
constexpr int kDenseMinRun = 16;                   // smallest dense_min accepted
constexpr int kDenseRunCap = TM_MAX_KP_LIMIT / kDenseMinRun;  // dense runs of a neighbour
constexpr int kDenseScan = 4;                      // query positions per thread and scan pass
constexpr int kDenseQcap = kDenseRows + kDenseScan * kDenseThreads;  // listed queries, at most
constexpr uint32_t kDenseTileBytes = 2048;         // 8 rows x 256 one-byte K values
constexpr uint32_t kDenseA = 0;                                          // 128 x 256 B
constexpr uint32_t kDenseB = kDenseA + kDenseRows / 8 * kDenseTileBytes;  // 128 x 256 B
constexpr uint32_t kDenseCol = kDenseB + kDenseCols / 8 * kDenseTileBytes;  // float4 (x, y, thr, -)
constexpr uint32_t kDensePart = kDenseCol + kDenseCols * 16;             // uint2 per row
constexpr uint32_t kDenseQlist = kDensePart + kDenseRows * 8;            // kDenseQcap u16
constexpr uint32_t kDenseRuns = kDenseQlist + kDenseQcap * 2;            // kDenseRunCap x (lo, hi) u16
constexpr uint32_t kDenseSmem = kDenseRuns + kDenseRunCap * 4;
// the neighbour's node keys are staged in the B area before the first tile
static_assert(kDenseCols / 8 * kDenseTileBytes >= TM_MAX_KP_LIMIT * 4, "B area holds the keys");
// > 1/4 of an SM's shared memory: at most three dense CTAs per SM, so their 3 x 128 columns
// never exceed the SM's 512 tensor-memory columns and an allocation cannot wait on a CTA that
// is not running
static_assert(4 * (kDenseSmem + 1024) > 233472, "dense CTAs must not exceed three per SM");

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A * B^T, A: M x 32 e4m3, B: N x 32 e4m3 (shared-memory descriptors).
__device__ __forceinline__ void tc_mma_e4m3(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Arrives once on bar when every tcgen05.mma this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// 16 consecutive accumulator columns of the warp's 32 lanes, then the wait (as tc_load32).
__device__ __forceinline__ void tc_load16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15])
                 :
                 : "memory");
}
// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16
// bytes; lbo = byte step between core matrices along K, sbo = along M (N); bit 46 = the
// descriptor version of this architecture.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo) {
    const uint64_t a = smem_addr(p);
    return ((a & 0x3FFFFull) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f8f6f4: float32 accumulator (bits 4-5 = 1), A and B e4m3
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_e4m3_f32(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// Four descriptor bits -> four e4m3 bytes, +1.0 (0x38) for a 0 bit, -1.0 (0xB8) for a 1 bit
// (the multiply moves bit i to bit 8i; the terms do not overlap, so nothing carries).
__device__ __forceinline__ uint32_t pm1_bytes(uint32_t x) {
    return (((x * 0x00204081u) & 0x01010101u) << 7) | 0x38383838u;
}
// Half h (descriptor bits 128h .. 128h + 127, one uint4) of row r of a K-major operand tile:
// bit k of the descriptor (32-bit word k / 32) at K index k; 8-row groups kDenseTileBytes
// apart, 16-byte K chunks 128 bytes apart within a group.
__device__ __forceinline__ void expand_half_row(unsigned char *tile, int r, int h, const uint4 &d) {
    const uint32_t w[4] = {d.x, d.y, d.z, d.w};
    unsigned char *row = tile + (r >> 3) * kDenseTileBytes + (r & 7) * 16 + h * 8 * 128;
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
        const uint32_t x = (w[kc >> 1] >> ((kc & 1) * 16)) & 0xFFFFu;
        *reinterpret_cast<uint4 *>(row + kc * 128) =
            make_uint4(pm1_bytes(x & 15u), pm1_bytes((x >> 4) & 15u), pm1_bytes((x >> 8) & 15u), pm1_bytes(x >> 12));
    }
}

__global__ void __launch_bounds__(kDenseThreads, 3) dense_kernel(BatchArgs A) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ float F[9];
    __shared__ float thr[kLevels], thre[kLevels], epl[2];
    __shared__ uint32_t wtot[32];
    __shared__ uint32_t s_taddr, s_fail;
    __shared__ __align__(8) uint64_t bar, never;
    unsigned char *sa = dsm + kDenseA, *sb = dsm + kDenseB;
    float4 *col = reinterpret_cast<float4 *>(dsm + kDenseCol);
    uint2 *part = reinterpret_cast<uint2 *>(dsm + kDensePart);
    uint16_t *qlist = reinterpret_cast<uint16_t *>(dsm + kDenseQlist);
    uint16_t *runs = reinterpret_cast<uint16_t *>(dsm + kDenseRuns);
    uint32_t *tkey = reinterpret_cast<uint32_t *>(sb);  // the neighbour's node keys, until the first tile
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int row = tid & (kDenseRows - 1), half = tid / kDenseRows;  // warps 4-7: second half
    const uint32_t splits = A.dsplit, item = blockIdx.x / splits, split = blockIdx.x % splits;
    const WorkItem w = A.items[item];
    if (A.sp.baseline_min_ratio > 0.0f) {  // (uniform) a skipped pair needs no dense blocks
        __shared__ bool s_skip;
        if (threadIdx.x == 0) s_skip = pair_skipped(w.pq, w.pt, w.mdepth, A.sp.baseline_min_ratio);
        __syncthreads();
        if (s_skip) return;
    }
    const KfView T = KfView::at(w.t, A.L);
    const int nQ = (int)w.nq, nT = (int)w.nt, dmin = A.sp.dense_min;
    for (int j0 = 0; j0 < nT; j0 += kDenseScan * kDenseThreads) {
        uint32_t v[kDenseScan];
#pragma unroll
        for (int u = 0; u < kDenseScan; ++u) {
            const int j = j0 + u * kDenseThreads + tid;
            v[u] = j < nT ? T.node[j] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kDenseScan; ++u) {
            const int j = j0 + u * kDenseThreads + tid;
            if (j < nT) tkey[j] = v[u];
        }
    }
    __syncthreads();
    // the neighbour's dense runs (node keys ascend), numbered in position order; this CTA
    // takes every splits-th
    const int per = (nT + kDenseThreads - 1) / kDenseThreads, jb = min(tid * per, nT), je = min(jb + per, nT);
    uint64_t starts = 0;  // bit j - jb: a dense run starts at j (per <= 32)
    for (int j = jb; j < je; ++j) {
        const uint32_t k = tkey[j];
        if ((j == 0 || tkey[j - 1] != k) && j + dmin - 1 < nT && tkey[j + dmin - 1] == k) starts |= 1ull << (j - jb);
    }
    uint32_t total;
    uint32_t r = block_scan_add((uint32_t)__popcll(starts), wtot, total);
    for (uint64_t m = starts; m; m &= m - 1) {
        const int j = jb + __ffsll((long long)m) - 1;
        if (r % splits == split) {
            runs[2 * (r / splits)] = (uint16_t)j;
            runs[2 * (r / splits) + 1] = (uint16_t)upper_bound_u32(tkey, j + dmin, nT, tkey[j]);
        }
        ++r;
    }
    const int nrun = total > split ? (int)((total - split + splits - 1) / splits) : 0;
    if (nrun == 0) return;  // uniform: total comes from the block scan
    if (wid == 0) {
        tmem_alloc(&s_taddr, kDenseCols);
        tmem_relinquish();
    }
    if (tid == 32) {
        mbar_init(&bar, 1);
        mbar_init(&never, 1);
        fence_mbar_init();
        s_fail = 0u;
    }
    // F and the epipole of the pair, as the prep kernel (which runs before this kernel) left them
    const float *pc = A.pconst + (size_t)kPairConst * w.idx;
    if (tid < 9) F[tid] = pc[tid];
    if (tid == 96 && A.sp.epipole_px > 0.0f) {
        epl[0] = pc[9];
        epl[1] = pc[10];
    }
    if (tid < kLevels) {
        const float sc = level_scale(tid);
        thr[tid] = fmul(A.sp.epi_chi2, fmul(sc, sc));
        thre[tid] = fmul(fmul(A.sp.epipole_px, A.sp.epipole_px), sc);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_taddr;
    const uint32_t tlane = tbase + ((uint32_t)((wid & 3) * 32) << 16);  // this warp's 32 lanes
    const bool epi = A.sp.epipolar != 0, eprej = A.sp.epipole_px > 0.0f;
    uint32_t phase = 0;
    for (int rr = 0; rr < nrun; ++rr) {
        const int lo = runs[2 * rr], hi = runs[2 * rr + 1];
        const uint32_t key = T.node[lo];
        const int ncol = hi - lo;
        bool b_ready = false;  // B operand of a one-tile run, kept over its query tiles
        // the node's eligible queries in ascending position: qlist[head .. qn) (uniform counts).
        // A stored query keyframe is in node-key order: the key's bucket bounds the scan.
        int scan = 0, head = 0, qn = 0, qend = nQ;
        if (!w.qraw) {
            const KfView Qv = KfView::at(w.q, A.L);
            const uint32_t b = key >> (32 - kBucketBits);
            scan = min((int)Qv.bstart[b], nQ);
            qend = min((int)Qv.bstart[b + 1], nQ);
        }
        for (;;) {
            if (qn - head < kDenseRows && scan < qend) {
                const int rest = qn - head;  // < 128: at most one entry per thread to move
                const uint16_t v = tid < rest ? qlist[head + tid] : (uint16_t)0;
                __syncthreads();
                if (tid < rest) qlist[tid] = v;
                qn = rest;
                head = 0;
                while (qn < kDenseRows && scan < qend) {
                    uint32_t nk[kDenseScan];
#pragma unroll
                    for (int u = 0; u < kDenseScan; ++u) {
                        const int p = scan + u * kDenseThreads + tid;
                        nk[u] = p < qend ? w.qnode[p] : 0u;
                    }
                    unsigned m[kDenseScan];
#pragma unroll
                    for (int u = 0; u < kDenseScan; ++u) {
                        const int p = scan + u * kDenseThreads + tid;
                        bool f = p < qend && (w.qraw ? node_key(nk[u]) : nk[u]) == key;
                        if (f && w.a != kNone)
                            f = A.masks[w.a + (w.qorig ? (uint32_t)w.qorig[p] : (uint32_t)p)] != 0;
                        m[u] = __ballot_sync(kFull, f);
                    }
                    if (lane == 0)
#pragma unroll
                        for (int u = 0; u < kDenseScan; ++u) wtot[u * 8 + wid] = (uint32_t)__popc(m[u]);
                    __syncthreads();
                    // entries in (pass u, warp, lane) order = ascending position
                    uint32_t run = (uint32_t)qn;
#pragma unroll
                    for (int u = 0; u < kDenseScan; ++u) {
                        uint32_t before = run;
                        for (int k = 0; k < kDenseThreads / 32; ++k) {
                            const uint32_t c = wtot[u * 8 + k];
                            if (k < wid) before += c;
                            run += c;
                        }
                        if ((m[u] >> lane) & 1u)
                            qlist[before + __popc(m[u] & ((1u << lane) - 1u))] = (uint16_t)(scan + u * kDenseThreads + tid);
                    }
                    qn = (int)run;
                    scan += kDenseScan * kDenseThreads;
                    __syncthreads();
                }
            }
            const int rows = min(qn - head, kDenseRows);
            if (rows == 0) break;  // every position scanned and every listed query done
            const bool mine = row < rows;
            const int p = mine ? guard((int)qlist[head + row], (int)w.nq, 18) : 0;
            Line l{};
            float den = 0.0f;
            uint32_t bk = kNone, sc = 0xFFFFu;
            if (mine) {
                const float2 xq = w.qxy[p];
                l = epi_line(F, xq.x, xq.y);
                den = epi_den(l);
                expand_half_row(sa, row, half, w.qdesc[2 * p + half]);
            }
            for (int n0 = 0; n0 < ncol; n0 += kDenseCols) {
                const int nc = min(kDenseCols, ncol - n0), nmma = (nc + 15) & ~15;
                if (!b_ready) {
                    if (row < nc) {
                        const int j = lo + n0 + row;
                        expand_half_row(sb, row, half, T.desc[2 * j + half]);
                        if (half == 0) {
                            const float2 xy = T.xy[j];
                            const bool e = w.b == kNone || A.masks[w.b + T.orig[j]] != 0;
                            const int lv = T.level[j];
                            col[row] = make_float4(xy.x, xy.y, e ? thr[lv] : -1.0f, thre[lv]);
                        }
                    }
                    b_ready = ncol <= kDenseCols;
                }
                fence_proxy_async();  // operand writes -> the tensor cores' reads
                __syncthreads();
                if (!s_fail) {
                    if (tid == 0) {
                        tc_fence_after();
                        const uint32_t idesc = idesc_e4m3_f32(kDenseRows, nmma);
#pragma unroll
                        for (int k = 0; k < 8; ++k)  // K = 256 bits in steps of 32
                            tc_mma_e4m3(tbase, smem_desc(sa + 256 * k, 128, kDenseTileBytes),
                                        smem_desc(sb + 256 * k, 128, kDenseTileBytes), idesc, k > 0);
                        tc_commit(&bar);
                    }
                    bool ok = mbar_wait_bounded(&bar, phase, A.wait_limit);
                    if (ok && A.starve) ok = mbar_wait_bounded(&never, 0, A.wait_limit);
                    phase ^= 1u;
                    if (!ok) s_fail = 1u;
                    tc_fence_before();
                    __syncthreads();
                    tc_fence_after();
                    if (!s_fail) {
                        // this warp's half of the columns (split in 16-column steps), 16 at a time
                        const int mid = ((nmma / 16 + 1) / 2) * 16;
                        for (int c0 = half ? mid : 0; c0 < (half ? nmma : mid); c0 += 16) {
                            uint32_t v[16];
                            tc_load16(tlane + (uint32_t)c0, v);
                            if (mine) {
#pragma unroll
                                for (int k = 0; k < 16; ++k) {
                                    const int c = c0 + k;
                                    const int dot = (int)__int_as_float(v[k]);
                                    const uint32_t d = (uint32_t)(256 - dot) >> 1;
                                    // an entry farther than the query's current second changes
                                    // neither its best nor its second: its gates are not needed
                                    if (c < nc && d <= sc) {
                                        const float4 cc = col[c];
                                        if (cc.z >= 0.0f && (!epi || epi_pass_den(l, den, cc.x, cc.y, cc.z)) &&
                                            !(eprej && near_epipole(epl, cc.x, cc.y, cc.w))) {
                                            const uint32_t kk = (d << 16) | (uint32_t)(lo + n0 + c);
                                            sc = min(sc, max(bk, kk) >> 16);
                                            bk = min(bk, kk);
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncthreads();  // accumulator and operands free for the next tile
            }
            // the two column halves of each query: merged by the first
            if (half == 1 && mine) part[row] = make_uint2(bk, sc);
            __syncthreads();
            if (half == 0 && mine) {
                const uint2 o = part[row];
                merge_best2(bk, sc, o.x, o.y);
                A.dres[w.c + (uint32_t)p] = s_fail ? make_uint2(kNone, kNone) : make_uint2(bk, sc);
            }
            head += rows;
        }
    }
    // after a wait that ran out, the tile's MMAs may still be in flight: wait for them (again
    // bounded) before the accumulator is released
    if (s_fail) mbar_wait_bounded(&bar, phase ^ 1u, A.wait_limit);
    tc_fence_before();
    __syncthreads();
    if (wid == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, kDenseCols);
    }
}


// One CTA per (new keyframe, neighbour) pair, largest pairs first (Sec. IV-C, all of S1-S6):
//   setup    the neighbour's node keys and bucket table into shared memory (bulk copies);
//            F by nine lanes of warp 0 (float64); winners reset; the neighbour's eligibility
//            read in node order (through the caller index of each position) and its eligible
//            positions listed with prefix counts (warp w takes a contiguous range of bitmap
//            words: ballots, one barrier, the list);
//   search   warps take 64-query groups (search_group), each accepted query listed with its
//            rotation bin;
//   finalize only the accepted queries are visited: kept if its target's winner, the top-3
//            rotation bins kept; a bitmap of the kept caller queries and its prefix counts give
//            every kept match its slot in caller query order.
// Comparisons (and a timed-out bulk copy) are recorded per item for the copy kernel.
// kMaxT: block size of the instance, 256 (five CTAs per SM) or 512 (two per SM: twice the warps
// on each pair, for batches of few pairs).
#ifndef TM_SEARCH_MINB
#define TM_SEARCH_MINB 5
#endif
constexpr int kSearchThreads = 256;
// The pair in slot `slot` of the launch order.  parity: phase of the CTA's bulk-copy barrier for
// this pair (the CTA's pairs alternate); first: the CTA's first pair (initializes the barriers).
// Returns 1 when a bounded wait ran out (the CTA stops).
// kForm: 0 the candidate rounds; 1 the entry form's join pass (the setup and the lookups, then
// the pair's entries listed for the evaluation pass; no finalize); 2 its finalize pass (the
// queries' states from the evaluation, then the results and finalize; a pair whose entries did
// not all fit is searched in rounds here instead).
template <int Q, bool kEpi, bool kEprej, bool kDense, bool kSplit, int kForm = 0>
__device__ __forceinline__ int search_pair(const BatchArgs &A, uint32_t slot, uint32_t parity, bool first) {
    constexpr int kMaxT = kSearchThreads;
    constexpr bool kLane = Q == 3;            // the per-lane form (two queries per lane)
    constexpr int QL = kLane ? 2 : Q;         // queries per lane of a group
    static_assert(!kLane || (!kEprej && !kDense), "the per-lane form runs the default gates");
    extern __shared__ __align__(128) unsigned char ssm[];
    __shared__ __align__(16) float thr[kLevels], thre[kLevels];
    __shared__ uint32_t qrec[kMaxT / 32][32 * QL], sbest[kMaxT / 32][32 * QL];  // per warp: its queries' states
    __shared__ uint32_t hist[32];
    __shared__ uint32_t keep, scmp, sdfail, nacc, s_last, sovf;
    __shared__ __align__(8) uint64_t bar, never;
    __shared__ int ok_all;
    constexpr int nw = kMaxT / 32;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const WorkItem w = A.sitems[slot];
    const uint32_t i = w.idx;
    const SearchStage S = SearchStage::make(A.sn);
    uint32_t *tkey = reinterpret_cast<uint32_t *>(ssm + S.tkey);
    uint16_t *bst = reinterpret_cast<uint16_t *>(ssm + S.bst);
    uint2 *words = reinterpret_cast<uint2 *>(ssm + S.words);
    uint16_t *epos = reinterpret_cast<uint16_t *>(ssm + S.epos);
    float *pc = reinterpret_cast<float *>(ssm + S.pc);
    uint32_t *win = reinterpret_cast<uint32_t *>(ssm + S.win);
    uint32_t *qbits = reinterpret_cast<uint32_t *>(ssm + S.qbits);
    uint32_t *qpre = reinterpret_cast<uint32_t *>(ssm + S.qpre);
    const KfView T = KfView::at(w.t, A.L);
    const int nQ = (int)w.nq, nT = (int)w.nt;
    const int nwq = (nQ + 31) >> 5, nwt = (nT + 31) >> 5;  // bitmap words: queries, targets
    // a split pair: this CTA takes part `part` of its query groups; the winners are global
    const int parts = kSplit && (int)(w.step >> 8) > 1 ? 2 : 1, part = parts > 1 ? (int)(w.step & 0xFFu) & 1 : 0;
    const int ngroups = (nQ + 32 * QL - 1) / (32 * QL), gpp = (ngroups + parts - 1) / parts;
    const int g0 = min(part * gpp, ngroups), g1 = min(g0 + gpp, ngroups);
    uint32_t *wing = parts > 1 ? A.pwin + w.toff : nullptr;
    const uint32_t abase = (uint32_t)(g0 * 32 * QL);
    static_assert(kForm == 0 || (!kLane && !kDense && !kEprej), "the entry form runs the default gates");
    if (kForm == 2 && (A.item_cmp[i] & kItemTimeout)) {  // (uniform) the join pass timed out
        if (tid == 0) A.counts[i] = 0u;
        return 0;
    }
    // the entry form's finalize of a pair whose entries all fit reads no staged tables
    const bool rounds = kForm != 2 || A.povf[i] != 0u;
    if (tid == 0) {
        // the neighbour's node keys and bucket table (store), its eligibility words and eligible
        // positions and the pair's constants (prep kernel), all into shared memory
        if (first) {
            mbar_init(&bar, 1);
            mbar_init(&never, 1);
            fence_mbar_init();
        }
        if (rounds) {
            const uint32_t kb = (4u * (uint32_t)nT + 15u) & ~15u;
            const uint32_t wb = (8u * (uint32_t)(nwt + 1) + 15u) & ~15u;
            const uint32_t eb = (2u * (uint32_t)nT + 15u) & ~15u;
            mbar_expect_tx(&bar, kb + (uint32_t)kBucketTableBytes + wb + eb + 48u);
            if (kb) bulk_g2s(tkey, T.node, kb, &bar);
            bulk_g2s(bst, T.bstart, (uint32_t)kBucketTableBytes, &bar);
            bulk_g2s(words, A.pwords + w.toff / 32u, wb, &bar);
            if (eb) bulk_g2s(epos, A.pepos + w.toff, eb, &bar);
            bulk_g2s(pc, A.pconst + (size_t)kPairConst * i, 48u, &bar);
        }
        scmp = 0u;
        sdfail = 0u;
        nacc = 0u;
        sovf = 0u;
        ok_all = 1;
    }
    if (tid == 32 && A.l2_prefetch && kForm == 0) {
        // the arrays the candidate rounds read, into L2 while the setup runs (each neighbour's
        // descriptors are read once, so their loads would otherwise wait on DRAM)
        bulk_prefetch_l2(T.desc, 32u * (uint32_t)nT);
        bulk_prefetch_l2(T.xy, (8u * (uint32_t)nT) & ~15u);
        bulk_prefetch_l2(w.qdesc, 32u * (uint32_t)nQ);
    }
    if (tid < kLevels) {
        const float sc = level_scale(tid);
        thr[tid] = fmul(A.sp.epi_chi2, fmul(sc, sc));
        thre[tid] = fmul(fmul(A.sp.epipole_px, A.sp.epipole_px), sc);
    }
    if (tid >= 96 && tid < 128) hist[tid - 96] = 0u;
    if (parts == 1)
        for (int j = tid; j < nT; j += kMaxT) win[j] = kNone;
    for (int k = tid; k < nwq; k += kMaxT) qbits[k] = 0u;
    QLoad<QL> cur = {};
    if (g0 + wid < g1) cur = load_group<QL>(A, w, g0 + wid);  // the first group's loads overlap the setup
    // the thread that initialized the barrier and issued the bulk copies awaits them; the CTA
    // barrier then publishes the copied data (and every other setup write) to all threads
    if (tid == 0 && rounds) {
        bool ok = mbar_wait_bounded(&bar, parity, A.wait_limit);
        if (ok && A.starve) ok = mbar_wait_bounded(&never, 0, A.wait_limit);
        if (!ok) ok_all = 0;
    }
    __syncthreads();
    if (!ok_all) {
        if (tid == 0) {
            A.counts[i] = 0u;
            if (kForm == 1) {
                // the finalize pass of the pair finds the flag and stops too
                if (parts > 1) atomicOr(A.item_cmp + i, kItemTimeout);
                else A.item_cmp[i] = kItemTimeout;
            } else if (parts > 1) {
                // the other part still counts this one in, and finds the pair failed
                A.pacc[2 * i + part] = 0u;
                atomicOr(A.item_cmp + i, kItemTimeout);
                __threadfence();
                atomicAdd(A.pdone + i, 1u);
            } else {
                A.item_cmp[i] = kItemTimeout;
            }
        }
        return 1;
    }
    if (A.sp.baseline_min_ratio > 0.0f &&
        (rounds ? pc[11] : A.pconst[(size_t)kPairConst * i + 11]) != 0.0f) {  // (uniform) pair-baseline skip
        if (tid == 0) {
            A.counts[i] = 0u;
            A.item_cmp[i] = 0u;
        }
        return 0;
    }
    SearchSmem M;
    M.tkey = smem_addr(tkey);
    M.bst = smem_addr(bst);
    M.words = smem_addr(words);
    M.epos = smem_addr(epos);
    M.win = smem_addr(win);
    M.pc = smem_addr(pc);
    M.thr = smem_addr(thr);
    M.thre = smem_addr(thre);
    M.rec = smem_addr(&qrec[wid][0]);
    M.sb = smem_addr(&sbest[wid][0]);
    uint32_t cmp = 0, dfail = 0;
    bool ovf = false;
    for (int g = g0 + wid; g < g1; g += nw) {
        QLoad<QL> nxt = {};
        if (g + nw < g1) nxt = load_group<QL>(A, w, g + nw);
        if constexpr (kLane)
            search_group_lane<kEpi>(A, w, T, M, &nacc, g, cur, cmp, wing, abase);
        else if constexpr (kForm == 1)
            join_group<QL>(A, w, M, g, cur, cmp, slot, ovf);
        else if (kForm == 2 && !rounds)
            final_group<QL>(A, w, T, M, &nacc, g, cur, dfail, wing, abase);
        else
            search_group<QL, kEpi, kEprej, kDense>(A, w, T, M, &nacc, g, cur, cmp, dfail, wing, abase);
        cur = nxt;
    }
    warp_count(cmp, &scmp);
    if (kForm == 1) {
        // the join pass ends here: the pair's comparisons (its entries) and overflow flag
        if (ovf) sovf = 1u;
        __syncthreads();
        if (tid == 0) {
            if (parts > 1) atomicAdd(A.item_cmp + i, scmp);
            else A.item_cmp[i] = scmp;
            if (sovf) A.povf[i] = 1u;
        }
        return 0;
    }
    if (kDense && __any_sync(kFull, dfail != 0u) && lane == 0) sdfail = 1u;
    if (parts > 1) __threadfence();  // (uniform) this thread's list entries and winners, device-wide
    __syncthreads();
    if (parts > 1) {
        // publish this part (its accepted list, winners, comparisons), then count it in: the
        // part that completes the count finalizes the pair (no CTA waits for another)
        if (tid == 0) {
            A.pacc[2 * i + part] = nacc;
            if (kForm == 0) atomicAdd(A.item_cmp + i, scmp);  // (the entry form's: by its join)
            if (sdfail) atomicOr(A.item_cmp + i, kItemTimeout);
            __threadfence();
            s_last = atomicAdd(A.pdone + i, 1u) == (uint32_t)(parts - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!s_last) return 0;
        __threadfence();
    }
    // finalize over the accepted queries (their list, written by this CTA, is read back from
    // L2 once; a thread keeps its first two entries in registers)
    // a split pair's lists: part 0's entries, then part 1's (read through L2: another CTA
    // wrote them)
    const int na0 = parts > 1 ? (int)__ldcg(A.pacc + 2 * i) : (int)nacc;
    const int na = parts > 1 ? na0 + (int)__ldcg(A.pacc + 2 * i + 1) : na0;
    const uint32_t abase1 = (uint32_t)(min(gpp, ngroups) * 32 * QL);
    const bool rot = A.sp.rot_filter != 0, res = A.sp.resolve != 0;
    auto load_entry = [&](int e) -> uint2 {
        if (parts == 1) return A.acc[w.c + (uint32_t)e];
        const uint32_t o = e < na0 ? (uint32_t)e : abase1 + (uint32_t)(e - na0);
        return __ldcg(A.acc + w.c + (uint32_t)guard((int)o, nQ, 20));
    };
    const uint2 v0 = tid < na ? load_entry(tid) : make_uint2(0u, 0u);
    const uint2 v1 = tid + kMaxT < na ? load_entry(tid + kMaxT) : make_uint2(0u, 0u);
    auto entry = [&](int e) -> uint2 {
        return e == tid ? v0 : (e == tid + kMaxT ? v1 : load_entry(e));
    };
    // a listed query is kept if it is its target's winner (io = caller index, j = target)
    auto winner = [&](const uint2 &v) -> bool {
        const uint32_t io = v.x & 0xFFFFu, j = (uint32_t)guard((int)(v.x >> 16), nT, 10);
        const uint32_t wv = parts > 1 ? __ldcg(wing + j) : win[j];
        return !res || wv == (((v.y >> 16) & 0x1FFu) << 16 | io);
    };
    if (rot)
        for (int e = tid; e < na; e += kMaxT) {
            const uint2 v = entry(e);
            if (winner(v)) atomicAdd(&hist[v.y >> 25], 1u);
        }
    __syncthreads();
    if (wid == 0) {
        const uint32_t k = rot ? top3_mask_warp(hist) : kNone;
        if (lane == 0) keep = k;
    }
    __syncthreads();
    const uint32_t kp = keep;
    for (int e = tid; e < na; e += kMaxT) {
        const uint2 v = entry(e);
        if (((kp >> (v.y >> 25)) & 1u) && winner(v)) {
            const uint32_t io = v.x & 0xFFFFu;
            atomicOr(&qbits[guard((int)(io >> 5), nwq, 11)], 1u << (io & 31u));
        }
    }
    __syncthreads();
    if (wid == 0) {
        // prefix counts of the bitmap's words: lane l takes words [l * pw, (l + 1) * pw)
        const int pw = (nwq + 31) >> 5, kb = min(lane * pw, nwq), ke = min(kb + pw, nwq);
        uint32_t s = 0;
        for (int k = kb; k < ke; ++k) s += (uint32_t)__popc(qbits[k]);
        uint32_t run = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, run, o);
            if (lane >= o) run += y;
        }
        run -= s;
        for (int k = kb; k < ke; ++k) {
            qpre[k] = run;
            run += (uint32_t)__popc(qbits[k]);
        }
        if (lane == 31) qpre[nwq] = run;
    }
    __syncthreads();
    const int lim = res ? min(nQ, nT) : nQ;
    for (int e = tid; e < na; e += kMaxT) {
        const uint2 v = entry(e);
        if (((kp >> (v.y >> 25)) & 1u) && winner(v)) {
            const uint32_t io = v.x & 0xFFFFu;
            const uint32_t r = qpre[io >> 5] + (uint32_t)__popc(qbits[io >> 5] & ((1u << (io & 31u)) - 1u));
            A.padded[w.out_off + (uint32_t)guard((int)r, lim, 12)] =
                Out3{(int)io, (int)(v.y & 0xFFFFu), (int)((v.y >> 16) & 0x1FFu)};
        }
    }
    if (tid == 0) {
        A.counts[i] = qpre[nwq];
        if (parts == 1 && kForm == 0) A.item_cmp[i] = scmp | (sdfail ? kItemTimeout : 0u);
    }
    return 0;
}

// The search kernel: one CTA per pair (grid = pairs), or, kPersist, CTAs that stay resident
// and take pairs in launch order (largest first) from the batch's work counter until none is
// left (the copy kernel resets the counter for the next run).
template <int Q, bool kEpi, bool kEprej, bool kDense, bool kPersist, bool kSplit = false, int kForm = 0>
__global__ void __launch_bounds__(kSearchThreads, TM_SEARCH_MINB) search_kernel(BatchArgs A) {
    __shared__ uint32_t s_slot;
    static_assert(kForm == 0 || !kPersist, "the entry form is not persistent");
    if (!kPersist) {
        search_pair<Q, kEpi, kEprej, kDense, kSplit, kForm>(A, blockIdx.x, 0u, true);
        return;
    }
    for (uint32_t it = 0;; ++it) {
        if (threadIdx.x == 0) s_slot = atomicAdd(A.work, 1u);
        __syncthreads();
        const uint32_t slot = s_slot;
        if (slot >= A.n_units) return;
        if (search_pair<Q, kEpi, kEprej, kDense, kSplit>(A, slot, it & 1u, it == 0)) return;
    }
}

// Per-pair preparation for the search kernel, one CTA per search item (Sec. IV-C pair setup).
// Warp 0: in every third CTA, F of that CTA's pair and the next two (float64, rounded to
// float32; nine lanes a pair, since this part's float64 pipe is narrow), then the epipole and
// the pair-baseline skip when those variants are on.  Warps 1 .. 7, meanwhile, the neighbour's
// eligibility in node order: each takes words [wb, we) of the position bitmap (a position's
// mask byte read through its caller index, four words' loads in flight per lane), records
// their ballots and counts, and after a barrier of these warps only writes each word with the
// eligible positions before it and lists its eligible positions, from the count of the warps
// before it; a closing word holds the total.
constexpr int kPrepThreads = 256;
__global__ void __launch_bounds__(kPrepThreads) pair_prep_kernel(BatchArgs A) {
    constexpr int nw = kPrepThreads / 32 - 1;  // eligibility warps (1 .. 7)
    __shared__ uint32_t wtot[nw];
    __shared__ float F3[3][12];
    __shared__ uint32_t sbits[TM_MAX_KP_LIMIT / 32];
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const uint32_t i = blockIdx.x;
    const WorkItem w = A.items[i];
    float *pc = A.pconst + (size_t)kPairConst * i;
    if (wid == 0) {
        // F of pairs 3 (i / 3) .. 3 (i / 3) + 2 by the first CTA of each three (one warp, 27 lanes)
        if (i % 3 == 0) {
            const double *tq[3], *tt[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const bool have = i + k < A.n_search;
                tq[k] = have ? A.items[i + k].pq : nullptr;
                tt[k] = have ? A.items[i + k].pt : nullptr;
            }
            fundamental_lanes3(A.cam, tq, tt, F3);
            __syncwarp();
            if (lane < 27 && i + lane / 9 < A.n_search)
                A.pconst[(size_t)kPairConst * (i + lane / 9) + lane % 9] = F3[lane / 9][lane % 9];
        }
        if (lane == 0) {
            float e[2] = {0.0f, 0.0f};
            if (A.sp.epipole_px > 0.0f) epipole_of(A.cam, w.pq, w.pt, e);
            pc[9] = e[0];
            pc[10] = e[1];
        }
        if (lane == 1)
            pc[11] = (A.sp.baseline_min_ratio > 0.0f && pair_skipped(w.pq, w.pt, w.mdepth, A.sp.baseline_min_ratio))
                         ? 1.0f : 0.0f;
        return;
    }
    const KfView T = KfView::at(w.t, A.L);
    const int nT = (int)w.nt, nwt = (nT + 31) >> 5;
    const int ew = wid - 1;  // eligibility warp index
    if ((w.step >> 8) > 1) {
        // a split pair: its global winners, its completion count and its comparison count
        // start over at every run
        for (int j = tid - 32; j < nT; j += kPrepThreads - 32) A.pwin[w.toff + (uint32_t)j] = kNone;
        if (tid == 32) {
            A.pdone[i] = 0u;
            A.item_cmp[i] = 0u;
        }
    }
    if (A.qpl == 4 && tid == 32) {
        // entry form: the pair's overflow flag and the batch's entry count start over every run
        A.povf[i] = 0u;
        if (i == 0) *A.nents = 0u;
    }
    uint2 *words = A.pwords + w.toff / 32u;
    uint16_t *epos = A.pepos + w.toff;
    const int per = (nwt + nw - 1) / nw, wb = min(ew * per, nwt), we = min(wb + per, nwt);
    uint32_t cnt = 0;
    constexpr int U = 4;
    for (int W0 = wb; W0 < we; W0 += U) {
        uint32_t o[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = 32 * (W0 + u) + lane;
            o[u] = (W0 + u < we && j < nT) ? (uint32_t)ldg(T.orig + j) : kNone;
        }
        bool m[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            m[u] = o[u] != kNone && (w.b == kNone || ldg(A.masks + w.b + o[u]) != 0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned bal = __ballot_sync(kFull, m[u]);
            if (W0 + u < we) {
                if (lane == 0) sbits[W0 + u] = bal;
                cnt += (uint32_t)__popc(bal);
            }
        }
    }
    if (lane == 0) wtot[ew] = cnt;
    asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");  // warps 1 .. 7 only
    uint32_t base = 0, ne = 0;
#pragma unroll
    for (int k = 0; k < nw; ++k) {
        const uint32_t v = wtot[k];
        if (k < ew) base += v;
        ne += v;
    }
    for (int W = wb; W < we; ++W) {
        const unsigned bal = sbits[W];
        if (lane == 0) words[W] = make_uint2(bal, base);
        if ((bal >> lane) & 1u) epos[base + (uint32_t)__popc(bal & ((1u << lane) - 1u))] = (uint16_t)(32 * W + lane);
        base += (uint32_t)__popc(bal);
    }
    if (tid == 32) words[nwt] = make_uint2(0u, ne);
}

// ---------------------------------------------------------------- fusion (S7-S9)

// One fusion item (up to kFuseChunk map points of a step) per CTA of 256 threads, thread t
// taking map points kFusePer t .. kFusePer t + kFusePer - 1 of the item.  The target keyframe's grid index,
// positions, caller indices and levels are bulk-copied into shared memory while each thread
// loads its two map points and runs their projection gates (which need only the target's
// pose); then each thread walks its map points' windows in shared memory and reads the
// descriptors of the keypoints that pass the reprojection gate; ordered compaction (map
// point order).
constexpr int kFuseThreads = 256;
constexpr int kFusePer = kFuseChunk / kFuseThreads;
static_assert(kFusePer * kFuseThreads == kFuseChunk, "whole map points per thread");
__global__ void __launch_bounds__(kFuseThreads) fuse_kernel(BatchArgs A) {
    extern __shared__ __align__(128) unsigned char fsm[];
    __shared__ FuseK K;
    __shared__ __align__(8) uint64_t bar, never;
    __shared__ uint32_t wtot[32];
    __shared__ uint32_t scmp;
    __shared__ bool ok_all;
    const int tid = threadIdx.x;
    const uint32_t item = A.n_search + blockIdx.x;
    if (item >= A.n_items) return;
    const WorkItem w = A.items[item];
    const SlotLayout &L = A.L;
    const FuseStage FS = FuseStage::make((int)A.fsn);
    const KfView Tg = KfView::at(w.q, L);
    const int nT = (int)w.nt;  // the target's keypoint count (set by the host)
    const uint32_t t16 = (uint32_t)((nT + 15) & ~15);
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init(&never, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, (uint32_t)(t16 * (8 + 2 + 2 + 1) + FuseStage::kGridStartBytes));
        bulk_g2s(fsm + FS.gstart, Tg.grid_start, (uint32_t)FuseStage::kGridStartBytes, &bar);
        if (t16) {
            bulk_g2s(fsm + FS.xy, Tg.xy, t16 * 8, &bar);
            bulk_g2s(fsm + FS.gitems, Tg.grid_items, t16 * 2, &bar);
            bulk_g2s(fsm + FS.orig, Tg.orig, t16 * 2, &bar);
            bulk_g2s(fsm + FS.level, Tg.level, t16, &bar);
        }
        scmp = 0u;
    }
    fuse_setup(Tg.hdr, A.fp.chi2, K);
    // the thread's map points: their loads overlap the staging
    bool have[kFusePer];
    float X[kFusePer], Y[kFusePer], Z[kFusePer], nx[kFusePer], ny[kFusePer], nz[kFusePer], mn[kFusePer],
        mx[kFusePer];
#pragma unroll
    for (int h = 0; h < kFusePer; ++h) {
        const uint32_t k = (uint32_t)(kFusePer * tid + h), m = w.a + k;
        have[h] = k < w.b && !(w.skip != kNone ? A.masks[w.skip + k] != 0 : (A.mp_skip && A.mp_skip[m]));
        const uint32_t mc = k < w.b ? m : w.a;  // (a valid index for the speculative loads)
        X[h] = A.mp_pos[3 * (size_t)mc];
        Y[h] = A.mp_pos[3 * (size_t)mc + 1];
        Z[h] = A.mp_pos[3 * (size_t)mc + 2];
        nx[h] = A.mp_normal[3 * (size_t)mc];
        ny[h] = A.mp_normal[3 * (size_t)mc + 1];
        nz[h] = A.mp_normal[3 * (size_t)mc + 2];
        mn[h] = A.mp_min[mc];
        mx[h] = A.mp_max[mc];
    }
    __syncthreads();  // K
    FuseProj P[kFusePer];
    bool pr[kFusePer];
    uint4 d[kFusePer][2];
#pragma unroll
    for (int h = 0; h < kFusePer; ++h) {
        pr[h] = have[h] && fuse_project(A.cam, A.fp, K, X[h], Y[h], Z[h], nx[h], ny[h], nz[h], mn[h], mx[h], P[h]);
        // the descriptor only of a map point that passed the gates
        const uint32_t mc = w.a + (uint32_t)(kFusePer * tid + h);
        d[h][0] = pr[h] ? A.mp_desc[2 * (size_t)mc] : make_uint4(0u, 0u, 0u, 0u);
        d[h][1] = pr[h] ? A.mp_desc[2 * (size_t)mc + 1] : make_uint4(0u, 0u, 0u, 0u);
    }
    const bool ok = staged_wait(&bar, &never, A);
    if (tid == 0) ok_all = true;
    __syncthreads();
    if (!ok) ok_all = false;
    __syncthreads();
    if (!ok_all) {
        if (tid == 0) {
            A.counts[item] = 0u;
            A.item_cmp[item] = kItemTimeout;
        }
        return;
    }
    KfView T = Tg;
    T.xy = reinterpret_cast<const float2 *>(fsm + FS.xy);
    T.grid_start = reinterpret_cast<const uint16_t *>(fsm + FS.gstart);
    T.grid_items = reinterpret_cast<const uint16_t *>(fsm + FS.gitems);
    T.orig = reinterpret_cast<const uint16_t *>(fsm + FS.orig);
    T.level = fsm + FS.level;
    uint32_t cmp = 0, r[kFusePer], nfound = 0;
#pragma unroll
    for (int h = 0; h < kFusePer; ++h) {
        r[h] = pr[h] ? fuse_window(T, nT, A.fp, K, P[h], d[h][0], d[h][1], cmp) : kNone;
        nfound += r[h] != kNone ? 1u : 0u;
    }
    warp_count(cmp, &scmp);
    uint32_t tot;
    uint32_t pos = block_scan_add(nfound, wtot, tot);
#pragma unroll
    for (int h = 0; h < kFusePer; ++h)
        if (r[h] != kNone) {
            const uint32_t m = w.a + (uint32_t)(kFusePer * tid + h);
            A.padded[w.out_off + (uint32_t)guard((int)pos, (int)w.b, 13)] =
                Out3{(int)(m - w.c), (int)(r[h] & 0xFFFFu), (int)(r[h] >> 16)};
            ++pos;
        }
    if (tid == 0) {
        A.counts[item] = tot;
        A.item_cmp[item] = scmp;
    }
}

// ---------------------------------------------------------------- triangulation (Map Point Creation)
//
// One CTA per pair, a thread per match of the pair's compacted list: parallax of the two
// viewing rays, the point as the midpoint of the rays' common perpendicular, depth and
// reprojection error in both views, scale consistency (Sec. III's constraints).  Float32 in a
// fixed order (dot products (x x' + y y') + z z'; this part's float64 rate is a small fraction
// of its float32 rate); the pose's R, t rounded from float64, its centre O = -R^T t formed in
// float64 and rounded.

struct TriView {
    float R[9], t[3], O[3];
};

__device__ __forceinline__ float dot3f(const float *a, const float *b) {
    return fadd(fadd(fmul(a[0], b[0]), fmul(a[1], b[1])), fmul(a[2], b[2]));
}

// depth and reprojection test of X in one view
__device__ __forceinline__ bool tri_view_ok(const TriView &v, const float *X, float fx, float fy, float cx,
                                            float cy, float u, float vv, float thr) {
    float c[3];
    for (int r = 0; r < 3; ++r)
        c[r] = fadd(fadd(fadd(fmul(v.R[r * 3 + 0], X[0]), fmul(v.R[r * 3 + 1], X[1])), fmul(v.R[r * 3 + 2], X[2])),
                    v.t[r]);
    if (!(c[2] > 0.0f)) return false;
    const float eu = fsub(fadd(fmul(fx, __fdiv_rn(c[0], c[2])), cx), u);
    const float ev = fsub(fadd(fmul(fy, __fdiv_rn(c[1], c[2])), cy), vv);
    return fadd(fmul(eu, eu), fmul(ev, ev)) <= thr;
}

__global__ void __launch_bounds__(128) tri_kernel(BatchArgs A) {
    __shared__ TriView V[2];
    __shared__ float sig2[kLevels], scl[kLevels];
    const uint32_t i = blockIdx.x;  // search item, logical order
    // (the search part's total follows the item offsets)
    const uint32_t o0 = A.offsets[i], o1 = A.offsets[i + 1 < A.n_search ? i + 1 : A.n_items];
    if (o0 == o1) return;
    const WorkItem w = A.items[i];
    const KfView Q = KfView::at(w.q, A.L), T = KfView::at(w.t, A.L);
    const int tid = threadIdx.x;
    if (tid < 2) {
        const double *P = tid == 0 ? Q.hdr->Tcw : T.hdr->Tcw;
        TriView &v = V[tid];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) v.R[r * 3 + c] = __double2float_rn(P[r * 4 + c]);
            v.t[r] = __double2float_rn(P[r * 4 + 3]);
        }
        for (int k = 0; k < 3; ++k) {
            double s = dmul(P[0 * 4 + k], P[0 * 4 + 3]);
            s = dadd(s, dmul(P[1 * 4 + k], P[1 * 4 + 3]));
            s = dadd(s, dmul(P[2 * 4 + k], P[2 * 4 + 3]));
            v.O[k] = __double2float_rn(-s);
        }
    }
    if (tid < kLevels) {
        const float sc = level_scale(tid);
        scl[tid] = sc;
        sig2[tid] = fmul(sc, sc);
    }
    __syncthreads();
    const float fx = __double2float_rn(A.cam.fx), fy = __double2float_rn(A.cam.fy);
    const float cx = __double2float_rn(A.cam.cx), cy = __double2float_rn(A.cam.cy);
    const float cos_max = __double2float_rn(A.tri_cos_max), chi2 = __double2float_rn(A.tri_chi2);
    const float fr = __double2float_rn(A.tri_ratio);
    for (uint32_t k = o0 + (uint32_t)tid; k < o1; k += blockDim.x) {
        const Out3 m = A.dense[k];
        // (q_idx, t_idx, dist) in caller order
        const int pq = guard(Q.pos[guard(m.a, (int)w.nq, 14)], (int)w.nq, 15);
        const int pt = guard(T.pos[guard(m.b, (int)w.nt, 16)], (int)w.nt, 17);
        const float2 xq = Q.xy[pq], xt = T.xy[pt];
        const int lev[2] = {Q.level[pq], T.level[pt]};
        const float u[2] = {xq.x, xt.x}, vv[2] = {xq.y, xt.y};
        float ray[2][3];
        for (int s = 0; s < 2; ++s) {
            const float xn = __fdiv_rn(fsub(u[s], cx), fx), yn = __fdiv_rn(fsub(vv[s], cy), fy);
            for (int c = 0; c < 3; ++c)
                ray[s][c] = fadd(fadd(fmul(V[s].R[0 * 3 + c], xn), fmul(V[s].R[1 * 3 + c], yn)), V[s].R[2 * 3 + c]);
        }
        float3 out = make_float3(0.0f, 0.0f, 0.0f);
        uint8_t ok = 0;
        const float a = dot3f(ray[0], ray[0]), b = dot3f(ray[0], ray[1]), c2 = dot3f(ray[1], ray[1]);
        const float cosp = __fdiv_rn(b, fmul(__fsqrt_rn(a), __fsqrt_rn(c2)));
        if (cosp > 0.0f && cosp < cos_max) {
            float wv[3];
            for (int q = 0; q < 3; ++q) wv[q] = fsub(V[0].O[q], V[1].O[q]);
            const float d = dot3f(ray[0], wv), e = dot3f(ray[1], wv);
            const float den = fsub(fmul(a, c2), fmul(b, b));
            if (den > 0.0f) {
                const float s1 = __fdiv_rn(fsub(fmul(b, e), fmul(c2, d)), den);
                const float s2 = __fdiv_rn(fsub(fmul(a, e), fmul(b, d)), den);
                float X[3];
                for (int q = 0; q < 3; ++q)
                    X[q] = fmul(fadd(fadd(V[0].O[q], fmul(s1, ray[0][q])), fadd(V[1].O[q], fmul(s2, ray[1][q]))), 0.5f);
                bool good = tri_view_ok(V[0], X, fx, fy, cx, cy, u[0], vv[0], fmul(chi2, sig2[lev[0]])) &&
                            tri_view_ok(V[1], X, fx, fy, cx, cy, u[1], vv[1], fmul(chi2, sig2[lev[1]]));
                if (good) {
                    float dist[2];
                    for (int s = 0; s < 2; ++s) {
                        float dv[3];
                        for (int q = 0; q < 3; ++q) dv[q] = fsub(X[q], V[s].O[q]);
                        dist[s] = __fsqrt_rn(dot3f(dv, dv));
                    }
                    good = dist[0] != 0.0f && dist[1] != 0.0f;
                    if (good) {
                        const float ratio_dist = __fdiv_rn(dist[1], dist[0]);
                        const float ratio_octave = __fdiv_rn(scl[lev[0]], scl[lev[1]]);
                        good = !(fmul(ratio_dist, fr) < ratio_octave || ratio_dist > fmul(ratio_octave, fr));
                    }
                }
                if (good) {
                    out = make_float3(X[0], X[1], X[2]);
                    ok = 1;
                }
            }
        }
        A.points[3 * (size_t)k] = out.x;
        A.points[3 * (size_t)k + 1] = out.y;
        A.points[3 * (size_t)k + 2] = out.z;
        A.point_ok[k] = ok;
    }
}

// Per-item counts -> offsets, and the per-item regions gathered into the dense output, for one
// part of the batch's items: part 0 the search items [0, n_search), launched on the search
// branch right after the search; part 1 the fusion items [n_search, n_items), on the store
// branch right after the fusion, its records from dense record out0 on (a fixed base past the
// search part's room), so that neither waits for the other branch.  Offsets are relative to
// the part's base; offsets[n_items + part] is the part's total.  Every CTA scans the part's
// counts itself (a few thousand words, read from L2 once into registers, kept with their
// offsets in shared memory), segment by segment, so that no CTA waits for another; CTA 0
// publishes the offsets, the part's comparison totals (search; fusion and forward fusion) and
// its status word (counters[2 + part]).  Warps copy items as 32-bit words (an output record is
// three words), so that a warp's loads and stores are contiguous.
constexpr int kCopyThreads = 1024;
constexpr int kCopyPer = 4;                          // counts per thread and segment
constexpr int kCopySeg = kCopyPer * kCopyThreads;    // items per scan segment
__global__ void __launch_bounds__(kCopyThreads) copy_kernel(BatchArgs A, uint32_t i0, uint32_t i1, uint32_t out0,
                                                             uint32_t part) {
    __shared__ uint32_t offs[kCopySeg], cnts[kCopySeg];
    __shared__ uint32_t wtot[32];
    const int tid = threadIdx.x, bs = blockDim.x;
    const uint32_t lane = tid & 31u, wid = tid >> 5, nw = bs >> 5;
    const uint32_t gw = blockIdx.x * nw + wid, gws = gridDim.x * nw;
    __shared__ unsigned long long csum[3][32];
    __shared__ uint32_t sflags;
    uint32_t base = 0;
    unsigned long long cs = 0, cf = 0, cw = 0;  // comparisons: search, fusion, forward fusion (CTA 0)
    uint32_t flags = 0;
    static_assert(sizeof(Out3) == 12, "three words per output record");
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(A.padded);
    uint32_t *dw = reinterpret_cast<uint32_t *>(A.dense + out0);
    for (uint32_t s0 = i0; s0 < i1; s0 += kCopySeg) {
        const uint32_t ns = min((uint32_t)kCopySeg, i1 - s0);
        // thread t takes items cb .. cb + kCopyPer - 1 of the segment (contiguous, so that the
        // prefix sum runs in item order)
        const uint32_t cb = (uint32_t)tid * kCopyPer;
        uint32_t c[kCopyPer], sum = 0;
#pragma unroll
        for (int q = 0; q < kCopyPer; ++q) {
            c[q] = cb + q < ns ? __ldg(A.counts + s0 + cb + q) : 0u;
            sum += c[q];
        }
        // the warp's first item of the segment: its count, region and first 128 words, loaded
        // before the scan so that their latency overlaps it
        const bool have0 = gw < ns;
        const uint32_t w0 = have0 ? 3u * __ldg(A.counts + s0 + gw) : 0u;
        const uint32_t src0 = have0 ? 3u * A.items[s0 + gw].out_off : 0u;
        uint32_t v0[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t e = 32u * q + lane;
            v0[q] = e < w0 ? __ldg(pw + src0 + e) : 0u;
        }
        if (blockIdx.x == 0)
#pragma unroll
            for (int q = 0; q < kCopyPer; ++q) {
                const uint32_t k = s0 + cb + q;
                if (cb + q >= ns) break;
                const uint32_t v = A.item_cmp[k];
                flags |= v & kItemTimeout;
                if (k < A.n_search) cs += v & ~kItemTimeout;
                else if (k < A.n_search + A.n_bwd) cf += v & ~kItemTimeout;
                else cw += v & ~kItemTimeout;
            }
        uint32_t total;
        uint32_t run = block_scan_add(sum, wtot, total) + base;
#pragma unroll
        for (int q = 0; q < kCopyPer; ++q)
            if (cb + q < ns) {
                offs[cb + q] = run;
                cnts[cb + q] = c[q];
                run += c[q];
            }
        __syncthreads();
        if (blockIdx.x == 0)
            for (uint32_t k = tid; k < ns; k += bs) A.offsets[s0 + k] = offs[k];
        for (uint32_t k = gw; k < ns; k += gws) {
            const bool first = k == gw;
            const uint32_t words = first ? w0 : 3u * cnts[k], dst = 3u * offs[k];
            const uint32_t src = first ? src0 : 3u * A.items[s0 + k].out_off;
            if (first) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t e = 32u * q + lane;
                    if (e < words) dw[dst + e] = v0[q];
                }
            }
            // four loads of each lane in flight before its stores
            for (uint32_t e0 = first ? 128u : 0u; e0 < words; e0 += 128) {
                uint32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t e = e0 + 32u * q + lane;
                    v[q] = e < words ? __ldg(pw + src + e) : 0u;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t e = e0 + 32u * q + lane;
                    if (e < words) dw[dst + e] = v[q];
                }
            }
        }
        base += total;
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            cs += __shfl_down_sync(kFull, cs, o);
            cf += __shfl_down_sync(kFull, cf, o);
            cw += __shfl_down_sync(kFull, cw, o);
        }
        flags = __reduce_or_sync(kFull, flags);
        if (tid == 0) sflags = 0u;
        if ((tid & 31) == 0) {
            csum[0][wid] = cs;
            csum[1][wid] = cf;
            csum[2][wid] = cw;
        }
        __syncthreads();
        if ((tid & 31) == 0 && flags) atomicOr(&sflags, flags);
        __syncthreads();
        if (tid == 0) {
            unsigned long long a = 0, b = 0, f = 0;
            for (uint32_t q = 0; q < nw; ++q) { a += csum[0][q]; b += csum[1][q]; f += csum[2][q]; }
            if (part == 0) {
                A.ncmp[0] = a;
                if (A.work) *A.work = 0u;  // the persistent search of the next run starts over
            } else {
                A.ncmp[1] = b;
                A.ncmp[2] = f;
            }
            A.counters[2 + part] = sflags ? kStatusTimeout : 0u;
            A.offsets[A.n_items + part] = base;
        }
    }
}

// ------------------------------------------------------------------------- integer-pipe rates
//
// Peak rates of the integer operations a descriptor comparison is made of, for the roofline's
// ALU term: every thread runs `iters` rounds over 8 independent register chains, so that
// throughput, not latency, bounds the launch.  mode 0: population count only (popc.b32);
// mode 1: three-input logic only (lop3.b32, xor of three); mode 2: one 256-bit Hamming
// distance per round (8 xor, 8 popc, the sum), operands in registers.  Inline PTX with
// volatile keeps every operation.  sink receives one word per thread so nothing is dead.
__global__ void __launch_bounds__(256) int_rate_kernel(int mode, int iters, uint32_t seed, uint32_t *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[8], y = seed ^ (t * 0x9E3779B1u), z = t + seed;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (t + 1u) * (2u * k + 1u) ^ seed;
    if (mode == 0) {
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("popc.b32 %0, %0;" : "+r"(x[k]));
    } else if (mode == 1) {
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[k]) : "r"(y), "r"(z));
    } else {
        uint32_t d = 0;
        for (int it = 0; it < iters; ++it) {
            uint32_t c[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                asm volatile("xor.b32 %0, %1, %2;" : "=r"(c[k]) : "r"(x[k]), "r"(y));
                asm volatile("popc.b32 %0, %0;" : "+r"(c[k]));
            }
            const uint32_t h = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
            d += h;
            y += h;  // the next round's operand depends on this one
        }
        x[0] = d;
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= x[k];
    sink[t] = r;
}

// ------------------------------------------------------------------------- plain form

// Stage 1: match.  One group of G lanes per sorted query; node ranges found by binary search
// in the neighbour's node array in global memory; winners per target by global atomicMin.
template <int G>
__global__ void pair_match_kernel(const unsigned char *qs, const unsigned char *ts,
                                  const uint8_t *mq, const uint8_t *mt, int cap, SearchConst sp,
                                  CamConst cam, PairScratch scr, unsigned long long *ncmp, float mdepth) {
    __shared__ float F[9];
    __shared__ float thr[kLevels], thre[kLevels], epl[2];
    __shared__ unsigned long long s_cmp;
    __shared__ bool s_skip;
    const SlotLayout L = SlotLayout::make(cap);
    const KfView Q = KfView::at(qs, L), T = KfView::at(ts, L);
    const int nQ = Q.hdr->n, nT = T.hdr->n;
    if (threadIdx.x < 32) fundamental_lanes(cam, Q.hdr->Tcw, T.hdr->Tcw, F);
    if (threadIdx.x == 32 && sp.epipole_px > 0.0f) epipole_of(cam, Q.hdr->Tcw, T.hdr->Tcw, epl);
    if (threadIdx.x == 64) s_skip = pair_skipped(Q.hdr->Tcw, T.hdr->Tcw, mdepth, sp.baseline_min_ratio);
    if (threadIdx.x == 0) s_cmp = 0ull;
    if (threadIdx.x < kLevels) {
        const float s = level_scale(threadIdx.x);
        thr[threadIdx.x] = fmul(sp.epi_chi2, fmul(s, s));
        thre[threadIdx.x] = fmul(fmul(sp.epipole_px, sp.epipole_px), s);
    }
    __syncthreads();
    const int g = threadIdx.x / G, sub = threadIdx.x % G;
    const int p = blockIdx.x * (blockDim.x / G) + g;
    uint32_t bkey = kNone, sec = 0xFFFFu;
    unsigned long long my_cmp = 0;
    if (p < nQ) {
        const uint32_t io = Q.orig[p];
        if (sub == 0) scr.res[io] = kNone;
        if (!s_skip && (!mq || mq[io])) {
            const uint32_t nd = Q.node[p];
            const int lo = lower_bound_u32(T.node, nT, nd);
            const int hi = (lo < nT && T.node[lo] == nd) ? upper_bound_u32(T.node, lo, nT, nd) : lo;
            if (lo < hi) {
                const uint4 q0 = Q.desc[2 * p], q1 = Q.desc[2 * p + 1];
                const float2 xq = Q.xy[p];
                const Line l = epi_line(F, xq.x, xq.y);
                for (int j = lo + sub; j < hi; j += G) {
                    if (mt && !mt[T.orig[j]]) continue;
                    ++my_cmp;
                    const uint32_t d = (uint32_t)hamming(q0, q1, T.desc[2 * j], T.desc[2 * j + 1]);
                    if (sp.epipolar || sp.epipole_px > 0.0f) {
                        const float2 xt = T.xy[j];
                        if (sp.epipolar && !epi_pass(l, xt.x, xt.y, thr[T.level[j]])) continue;
                        if (sp.epipole_px > 0.0f && near_epipole(epl, xt.x, xt.y, thre[T.level[j]])) continue;
                    }
                    const uint32_t key = (d << 16) | (uint32_t)j;
                    if (key < bkey) { sec = min(sec, bkey >> 16); bkey = key; }
                    else sec = min(sec, d);
                }
            }
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const uint32_t ob = __shfl_xor_sync(kFull, bkey, off);
        const uint32_t os = __shfl_xor_sync(kFull, sec, off);
        sec = min(min(sec, os), max(bkey, ob) >> 16);
        bkey = min(bkey, ob);
    }
    if (sub == 0 && p < nQ) {
        uint32_t acc = kNone;
        if (bkey != kNone) {
            const uint32_t best = bkey >> 16;
            bool ok = (int)best <= sp.hamming_max;
            if (ok && sp.ratio_num != 0 && sec != 0xFFFFu)
                ok = (long long)sp.ratio_den * best < (long long)sp.ratio_num * sec;
            if (ok) {
                const uint32_t j = bkey & 0xFFFFu;
                acc = (j << 16) | best;
                if (sp.resolve) atomicMin(&scr.win[j], (best << 16) | Q.orig[p]);
            }
        }
        scr.accq[p] = acc;
    }
    if (my_cmp) atomicAdd(&s_cmp, my_cmp);
    __syncthreads();
    if (threadIdx.x == 0 && s_cmp) atomicAdd(ncmp, s_cmp);
}

// Stage 2: keep the winner of every target, histogram the rotation of kept matches.
__global__ void pair_resolve_kernel(const unsigned char *qs, const unsigned char *ts, int cap,
                                    SearchConst sp, PairScratch scr) {
    const SlotLayout L = SlotLayout::make(cap);
    const KfView Q = KfView::at(qs, L), T = KfView::at(ts, L);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Q.hdr->n) return;
    const uint32_t acc = scr.accq[p];
    if (acc == kNone) return;
    const uint32_t j = acc >> 16, d = acc & 0xFFFFu, io = Q.orig[p];
    if (sp.resolve && scr.win[j] != ((d << 16) | io)) return;
    uint32_t bin = 0;
    if (sp.rot_filter) {
        bin = (uint32_t)rot_bin(Q.angle[p], T.angle[j], sp.rot_mode);
        atomicAdd(&scr.hist[bin], 1u);
    }
    scr.res[io] = pack_res(T.orig[j], d, bin);
}

// Stage 3 (one CTA): top-3 bins, ordered compaction appended at *running.
__global__ void pair_compact_kernel(const unsigned char *qs, int cap, SearchConst sp,
                                    PairScratch scr, Out3 *dense, uint32_t *pair_offset) {
    __shared__ uint32_t wtot[32];
    __shared__ uint32_t keep;
    const SlotLayout L = SlotLayout::make(cap);
    const KfView Q = KfView::at(qs, L);
    const int nQ = Q.hdr->n;
    if (threadIdx.x == 0) keep = sp.rot_filter ? top3_mask(scr.hist) : kNone;
    __syncthreads();
    const uint32_t start = *scr.running;
    uint32_t base = 0;
    for (int i0 = 0; i0 < nQ; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const uint32_t r = i < nQ ? scr.res[i] : kNone;
        const bool f = r != kNone && ((keep >> (r & 31u)) & 1u);
        uint32_t tot;
        const uint32_t pos = block_scan_flag(f, wtot, tot);
        if (f) dense[start + base + pos] = Out3{i, (int)(r >> 14), (int)((r >> 5) & 0x1FFu)};
        base += tot;
    }
    if (threadIdx.x == 0) {
        pair_offset[0] = start;
        *scr.running = start + base;
    }
}

__global__ void fuse_plain_kernel(const unsigned char *ts, int cap, const float *pos,
                                  const float *normal, const uint4 *desc, const float *mn,
                                  const float *mx, const uint8_t *skip, int n, FuseConst fp,
                                  CamConst cam, uint32_t *res, unsigned long long *ncmp) {
    __shared__ FuseK K;
    __shared__ uint32_t scmp;
    const SlotLayout L = SlotLayout::make(cap);
    const KfView T = KfView::at(ts, L);
    if (threadIdx.x == 0) scmp = 0u;
    fuse_setup(T.hdr, fp.chi2, K);
    __syncthreads();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cmp = 0;
    if (m < n) {
        uint32_t r = kNone;
        if (!(skip && skip[m]))
            r = fuse_one(T, T.hdr->n, cam, fp, K, load_mp(pos + 3 * (size_t)m, normal + 3 * (size_t)m,
                                                desc + 2 * (size_t)m, mn[m], mx[m]), cmp);
        res[m] = r;
    }
    warp_count(cmp, &scmp);
    __syncthreads();
    if (threadIdx.x == 0 && scmp) atomicAdd(ncmp, (unsigned long long)scmp);
}

__global__ void fuse_compact_kernel(const uint32_t *res, int n, Out3 *dense, uint32_t *running,
                                    uint32_t *offset_out) {
    __shared__ uint32_t wtot[32];
    const uint32_t start = *running;
    uint32_t base = 0;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const uint32_t r = i < n ? res[i] : kNone;
        uint32_t tot;
        const uint32_t pos = block_scan_flag(r != kNone, wtot, tot);
        if (r != kNone) dense[start + base + pos] = Out3{i, (int)(r & 0xFFFFu), (int)(r >> 16)};
        base += tot;
    }
    if (threadIdx.x == 0) {
        *offset_out = start;
        *running = start + base;
    }
}

}  // namespace

// ------------------------------------------------------------------------- launchers

size_t ingest_smem_bytes(int cap) { return 18 * ingest_pow2(cap); }

// Launch with a scheduling priority (cudaLaunchAttributePriority; kept by stream capture in
// the graph's kernel node): when SMs free up, CTAs of higher-priority kernels are placed
// first.  prio 0 = the stream's default.
template <typename... Args>
static cudaError_t launch_prio(void (*k)(Args...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               int prio, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = prio ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

cudaError_t launch_stage_gather(const GatherJob *jobs, int n, unsigned char *base, const size_t offs[5],
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    StageOffsets o;
    for (int q = 0; q < 5; ++q) o.o[q] = offs[q];
    stage_gather_kernel<<<n, 256, 0, s>>>(jobs, base, o);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestArgs &a, cudaStream_t s, int prio) {
    if (a.n_jobs <= 0) return cudaSuccess;
    const size_t smem = ingest_smem_bytes(a.cap);
    cudaError_t e = cudaFuncSetAttribute(ingest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return launch_prio(ingest_kernel, dim3(a.n_jobs), dim3(kIngestThreads), smem, s, prio, a);
}

size_t search_smem_bytes(int sn) { return SearchStage::make(sn).bytes; }

// The search kernel instance for a launch: the group form (rounds with 1 or 2 queries per lane,
// or 3: the per-lane form) and the persistent form exist for the gate configurations of the
// default search (epipolar gate on
// or off, no epipole rejection, no dense blocks); any other configuration runs 64-query groups,
// one CTA per pair (search_form reports the form a launch gets).
static bool search_variants(const BatchArgs &a) { return !(a.sp.epipole_px > 0.0f) && !(a.sp.dense_min > 0); }
// The entry form's join (kForm 1) and finalize (kForm 2) instances.
static void (*entry_fn(const BatchArgs &a, int form))(BatchArgs) {
    const bool epi = a.sp.epipolar != 0, split = a.n_units > a.n_search;
    if (form == 1)
        return split ? (epi ? search_kernel<2, true, false, false, false, true, 1> : search_kernel<2, false, false, false, false, true, 1>)
                     : (epi ? search_kernel<2, true, false, false, false, false, 1> : search_kernel<2, false, false, false, false, false, 1>);
    return split ? (epi ? search_kernel<2, true, false, false, false, true, 2> : search_kernel<2, false, false, false, false, true, 2>)
                 : (epi ? search_kernel<2, true, false, false, false, false, 2> : search_kernel<2, false, false, false, false, false, 2>);
}

static void (*search_fn(const BatchArgs &a))(BatchArgs) {
    const bool epi = a.sp.epipolar != 0, eprej = a.sp.epipole_px > 0.0f, dense = a.sp.dense_min > 0;
    if (search_variants(a) && a.qpl == 4) return entry_fn(a, 2);
    if (search_variants(a) && a.n_units > a.n_search) {  // split pairs: their own instances
        if (a.qpl == 3) return epi ? search_kernel<3, true, false, false, false, true> : search_kernel<3, false, false, false, false, true>;
        if (a.qpl == 1) return epi ? search_kernel<1, true, false, false, false, true> : search_kernel<1, false, false, false, false, true>;
        return epi ? search_kernel<2, true, false, false, false, true> : search_kernel<2, false, false, false, false, true>;
    }
    if (search_variants(a)) {
        if (a.qpl == 3 && !a.persist)
            return epi ? search_kernel<3, true, false, false, false> : search_kernel<3, false, false, false, false>;
        if (a.qpl == 1)
            return a.persist ? (epi ? search_kernel<1, true, false, false, true> : search_kernel<1, false, false, false, true>)
                             : (epi ? search_kernel<1, true, false, false, false> : search_kernel<1, false, false, false, false>);
        return a.persist ? (epi ? search_kernel<2, true, false, false, true> : search_kernel<2, false, false, false, true>)
                         : (epi ? search_kernel<2, true, false, false, false> : search_kernel<2, false, false, false, false>);
    }
    if (dense) {
        if (epi) return eprej ? search_kernel<2, true, true, true, false> : search_kernel<2, true, false, true, false>;
        return eprej ? search_kernel<2, false, true, true, false> : search_kernel<2, false, false, true, false>;
    }
    return epi ? search_kernel<2, true, true, false, false> : search_kernel<2, false, true, false, false>;
}

void search_form(BatchArgs &a) {
    if (!search_variants(a)) {
        a.qpl = 2;
        a.persist = 0;
    }
    if (a.qpl == 3 || a.qpl == 4) a.persist = 0;  // the per-lane and entry forms have no persistent instance
    if (a.n_units > a.n_search) a.persist = 0;  // nor do split pairs
}

int search_ctas_per_sm(const BatchArgs &a) {
    int n = 0;
    const size_t smem = search_smem_bytes(a.sn);
    if (cudaFuncSetAttribute(search_fn(a), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) return 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_fn(a), kSearchThreads, smem) == cudaSuccess ? n : 0;
}

cudaError_t launch_prep(const BatchArgs &a, cudaStream_t s, int prio) {
    if (a.n_search == 0) return cudaSuccess;
    return launch_prio(pair_prep_kernel, dim3(a.n_search), dim3(kPrepThreads), 0, s, prio, a);
}

cudaError_t launch_search(const BatchArgs &a, int ctas, cudaStream_t s, int prio) {
    if (a.n_search == 0) return cudaSuccess;
    const size_t smem = search_smem_bytes(a.sn);
    cudaError_t e = cudaFuncSetAttribute(search_fn(a), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.qpl == 4 && search_variants(a)) {
        // the entry form: join (one CTA per launch entry), evaluation (a grid stride over the
        // entries, eight CTAs per SM), finalize (one CTA per launch entry)
        void (*join)(BatchArgs) = entry_fn(a, 1), (*fin)(BatchArgs) = entry_fn(a, 2);
        static int sms = 0;
        if (!sms) {
            int d = 0;
            if ((e = cudaGetDevice(&d)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d)))
                return e;
        }
        if ((e = cudaFuncSetAttribute(join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
            (e = launch_prio(join, dim3(a.n_units), dim3(kSearchThreads), smem, s, prio, a)))
            return e;
        void (*ev)(BatchArgs) = a.sp.epipolar ? eval_kernel<true> : eval_kernel<false>;
        if ((e = launch_prio(ev, dim3(8 * sms), dim3(kEvalThreads), 0, s, prio, a))) return e;
        return launch_prio(fin, dim3(a.n_units), dim3(kSearchThreads), smem, s, prio, a);
    }
    const uint32_t grid = a.persist ? (uint32_t)std::max(1, std::min(ctas, (int)a.n_units)) : a.n_units;
    return launch_prio(search_fn(a), dim3(grid), dim3(kSearchThreads), smem, s, prio, a);
}

size_t dense_smem_bytes() { return kDenseSmem; }

cudaError_t launch_dense(const BatchArgs &a, cudaStream_t s, int prio) {
    if (a.n_search == 0 || a.sp.dense_min <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem);
    if (e != cudaSuccess) return e;
    return launch_prio(dense_kernel, dim3(a.n_search * a.dsplit), dim3(kDenseThreads), kDenseSmem, s, prio, a);
}

cudaError_t launch_fuse(const BatchArgs &a, cudaStream_t s, int prio) {
    const uint32_t blocks = a.n_items - a.n_search;
    if (blocks == 0) return cudaSuccess;
    const size_t smem = FuseStage::make((int)a.fsn).bytes;
    cudaError_t e = cudaFuncSetAttribute(fuse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_prio(fuse_kernel, dim3(blocks), dim3(kFuseThreads), smem, s, prio, a);
}

cudaError_t launch_tri(const BatchArgs &a, cudaStream_t s) {
    if (!a.triangulate || a.n_search == 0) return cudaSuccess;
    tri_kernel<<<a.n_search, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t debug_bounds(bool reset, uint32_t *site, bool *enabled) {
#ifdef TM_DEBUG_BOUNDS
    *enabled = true;
    cudaError_t e = cudaMemcpyFromSymbol(site, g_bounds_site, sizeof(uint32_t));
    if (e == cudaSuccess && reset) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_bounds_site, &zero, sizeof zero);
    }
    return e;
#else
    (void)reset;
    *enabled = false;
    *site = 0u;
    return cudaSuccess;
#endif
}

cudaError_t launch_int_rate(int mode, int ctas, int iters, uint32_t *sink, cudaStream_t s) {
    int_rate_kernel<<<ctas, 256, 0, s>>>(mode, iters, 0x1234567u, sink);
    return cudaGetLastError();
}

cudaError_t launch_copy(const BatchArgs &a, int part, uint32_t out0, int ctas, cudaStream_t s) {
    const uint32_t i0 = part == 0 ? 0u : a.n_search, i1 = part == 0 ? a.n_search : a.n_items;
    if (i0 >= i1) return cudaSuccess;
    copy_kernel<<<ctas, kCopyThreads, 0, s>>>(a, i0, i1, out0, (uint32_t)part);
    return cudaGetLastError();
}

size_t pair_scratch_bytes(int cap) { return align128(size_t(cap) * 4) * 3 + 256; }

PairScratch pair_scratch_at(void *base, int cap) {
    unsigned char *b = static_cast<unsigned char *>(base);
    const size_t a = align128(size_t(cap) * 4);
    PairScratch s;
    s.win = reinterpret_cast<uint32_t *>(b);
    s.accq = reinterpret_cast<uint32_t *>(b + a);
    s.res = reinterpret_cast<uint32_t *>(b + 2 * a);
    s.hist = reinterpret_cast<uint32_t *>(b + 3 * a);
    s.running = reinterpret_cast<uint32_t *>(b + 3 * a + 128);
    return s;
}

cudaError_t launch_pair_plain(const unsigned char *q, const unsigned char *t, const uint8_t *mq,
                              const uint8_t *mt, int nq, int nt, int cap, const SearchConst &sp,
                              const CamConst &cam, const PairScratch &scr, Out3 *dense,
                              uint32_t *pair_offset, unsigned long long *ncmp, int lanes,
                              cudaStream_t s, float t_median_depth) {
    cudaError_t e;
    if (nt > 0 && (e = cudaMemsetAsync(scr.win, 0xFF, size_t(nt) * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(scr.hist, 0, 128, s)) != cudaSuccess) return e;
    const int threads = 256;
    if (nq > 0) {
        const int per = threads / lanes;
        const int grid = (nq + per - 1) / per;
        switch (lanes) {
            case 1: pair_match_kernel<1><<<grid, threads, 0, s>>>(q, t, mq, mt, cap, sp, cam, scr, ncmp, t_median_depth); break;
            case 2: pair_match_kernel<2><<<grid, threads, 0, s>>>(q, t, mq, mt, cap, sp, cam, scr, ncmp, t_median_depth); break;
            case 4: pair_match_kernel<4><<<grid, threads, 0, s>>>(q, t, mq, mt, cap, sp, cam, scr, ncmp, t_median_depth); break;
            case 8: pair_match_kernel<8><<<grid, threads, 0, s>>>(q, t, mq, mt, cap, sp, cam, scr, ncmp, t_median_depth); break;
            case 16: pair_match_kernel<16><<<grid, threads, 0, s>>>(q, t, mq, mt, cap, sp, cam, scr, ncmp, t_median_depth); break;
            default: pair_match_kernel<32><<<grid, threads, 0, s>>>(q, t, mq, mt, cap, sp, cam, scr, ncmp, t_median_depth); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        pair_resolve_kernel<<<(nq + 255) / 256, 256, 0, s>>>(q, t, cap, sp, scr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    pair_compact_kernel<<<1, 1024, 0, s>>>(q, cap, sp, scr, dense, pair_offset);
    return cudaGetLastError();
}

cudaError_t launch_fuse_plain(const unsigned char *t, int cap, const float *pos,
                              const float *normal, const uint4 *desc, const float *mn,
                              const float *mx, const uint8_t *skip, int n, const FuseConst &fp,
                              const CamConst &cam, uint32_t *res, Out3 *dense, uint32_t *running,
                              uint32_t *offset_out, unsigned long long *ncmp, cudaStream_t s) {
    if (n > 0) {
        fuse_plain_kernel<<<(n + 255) / 256, 256, 0, s>>>(t, cap, pos, normal, desc, mn, mx, skip,
                                                          n, fp, cam, res, ncmp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    fuse_compact_kernel<<<1, 1024, 0, s>>>(res, n, dense, running, offset_out);
    return cudaGetLastError();
}

}  // namespace tmap

// ------------------------------------------------------------------------- no-allocation variant
//
// Some callers cannot allocate device memory: code under an allocator that must not grow (a
// fixed memory budget), a real-time loop that forbids allocation after start-up (an
// allocation may block or synchronise the device), or a host without a tm_ctx and its store.
// For them tm_search_pair_noalloc searches one keyframe pair with the plain per-pair kernels,
// keeping all of its scratch -- the two node-sorted keyframe slots, the per-pair arrays and
// the counters -- in the file-scope array below, which every GPU that loads the library holds
// until the process exits.

#include "runtime.h"

namespace {

constexpr int kNoAllocMaxKp = TM_NOALLOC_MAX_KP;
constexpr size_t kNoAllocSlot = tmap::SlotLayout::make(kNoAllocMaxKp).bytes;
constexpr size_t kNoAllocPair = tmap::align128(size_t(kNoAllocMaxKp) * 4) * 3 + 256;
// [slot Q | slot T | pair scratch | two ingest jobs | n_comparisons]
constexpr size_t kNoAllocJobs = 2 * kNoAllocSlot + kNoAllocPair;
constexpr size_t kNoAllocCmp = kNoAllocJobs + tmap::align128(2 * sizeof(tmap::IngestJob));
constexpr size_t kNoAllocBytes = kNoAllocCmp + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Writes the two ingest jobs (passed by value) into the scratch array.
__global__ void noalloc_jobs_kernel(tmap::IngestJob *dst, tmap::IngestJob q, tmap::IngestJob t) {
    dst[0] = q;
    dst[1] = t;
}

// Device address of the scratch array for the current device, looked up once per device (the
// first call with that device current) and kept for the life of the process.  A device reset
// (cudaDeviceReset) while the library is loaded would leave the kept address stale.
// (In host code g_noalloc_scratch names a host-side stand-in, not device memory.)
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[64] = {nullptr};

tm_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= 64) return tmap::fail(TM_ERR_INVALID_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return tmap::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[device];
    return TM_OK;
}

// p is memory the kernels on `device` read directly: device memory of that device (or managed
// memory), aligned to `align` bytes (the width of the kernels' loads and stores).
bool device_accessible(const void *p, int device, size_t align) {
    if (reinterpret_cast<uintptr_t>(p) % align) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" tm_status tm_search_pair_noalloc(const tm_camera *cam, const tm_keyframe_view *q,
                                            const tm_keyframe_view *t,
                                            const tm_search_params *params,
                                            const uint8_t *q_free, const uint8_t *t_free,
                                            tm_match *out, uint32_t *n_out,
                                            uint64_t *n_comparisons, void *stream) {
    using namespace tmap;
    if (!cam || !q || !t || !out || !n_out)
        return fail(TM_ERR_INVALID_ARG, "tm_search_pair_noalloc: null argument");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > TM_MAX_IMAGE_SIZE ||
        cam->height > TM_MAX_IMAGE_SIZE || !(cam->fx > 0) || !(cam->fy > 0))
        return fail(TM_ERR_INVALID_ARG, "tm_search_pair_noalloc: bad camera (image sides 1..%d px, fx, fy > 0)",
                    TM_MAX_IMAGE_SIZE);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    for (const tm_keyframe_view *v : {q, t}) {
        if (v->n < 0 || v->n > kNoAllocMaxKp)
            return fail(TM_ERR_INVALID_ARG,
                        "tm_search_pair_noalloc: %d keypoints exceed the limit of %d per keyframe "
                        "(the size of the library's fixed scratch array)", v->n, kNoAllocMaxKp);
        if (v->n > 0 && !(device_accessible(v->desc, dev, 16) && device_accessible(v->xy, dev, 8) &&
                          device_accessible(v->angle, dev, 4) && device_accessible(v->level, dev, 1) &&
                          device_accessible(v->node, dev, 4)))
            return fail(TM_ERR_INVALID_ARG,
                        "tm_search_pair_noalloc: keyframe arrays must be memory of the current device "
                        "(desc 16-byte, xy 8-byte, angle and node 4-byte aligned)");
    }
    if (!device_accessible(out, dev, 4) || !device_accessible(n_out, dev, 4) ||
        (n_comparisons && !device_accessible(n_comparisons, dev, 8)) ||
        (q_free && !device_accessible(q_free, dev, 1)) || (t_free && !device_accessible(t_free, dev, 1)))
        return fail(TM_ERR_INVALID_ARG,
                    "tm_search_pair_noalloc: masks and outputs must be memory of the current device "
                    "(out and n_out 4-byte, n_comparisons 8-byte aligned)");
    tm_search_params sp;
    tm_search_params_default(&sp);
    if (params) sp = *params;
    if (sp.hamming_max < 0 || sp.ratio_num < 0 || sp.ratio_den < 0 || !(sp.epi_chi2 >= 0) ||
        !(sp.epipole_px >= 0.0f && sp.epipole_px < 1e6f) || (sp.rot_mode != 0 && sp.rot_mode != 1))
        return fail(TM_ERR_INVALID_ARG, "tm_search_pair_noalloc: bad search parameters");
    const int l = sp.lanes_per_query ? sp.lanes_per_query : 1;
    if (!(l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32))
        return fail(TM_ERR_INVALID_ARG, "tm_search_pair_noalloc: bad lanes_per_query");
    unsigned char *scr = nullptr;
    tm_status st = noalloc_scratch(dev, &scr);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *slot_q = scr, *slot_t = scr + kNoAllocSlot;
    PairScratch ps = pair_scratch_at(scr + 2 * kNoAllocSlot, kNoAllocMaxKp);
    IngestJob *jobs = reinterpret_cast<IngestJob *>(scr + kNoAllocJobs);
    unsigned long long *ncmp = reinterpret_cast<unsigned long long *>(scr + kNoAllocCmp);
    // the scratch keeps the previous call's contents: clear what must start at zero
    if ((e = cudaMemsetAsync(ps.running, 0, 8, s)) || (e = cudaMemsetAsync(ncmp, 0, 8, s)))
        return cuda_fail(e, "scratch reset");
    IngestJob jq{}, jt{};
    jq.slot = slot_q;
    jq.src = 0;
    jq.n = q->n;
    jt.slot = slot_t;
    jt.src = 0;
    jt.n = t->n;
    for (int k = 0; k < 12; ++k) {
        jq.Tcw[k] = q->Tcw[k];
        jt.Tcw[k] = t->Tcw[k];
    }
    noalloc_jobs_kernel<<<1, 1, 0, s>>>(jobs, jq, jt);
    if ((e = cudaGetLastError())) return cuda_fail(e, "job kernel");
    const CamConst cc = CamConst::make(cam->fx, cam->fy, cam->cx, cam->cy, cam->width, cam->height);
    const tm_keyframe_view *views[2] = {q, t};
    for (int k = 0; k < 2; ++k) {  // node order and grid of each keyframe, into its scratch slot
        IngestArgs a;
        a.jobs = jobs + k;
        a.n_jobs = 1;
        a.cap = kNoAllocMaxKp;
        a.desc = reinterpret_cast<const uint4 *>(views[k]->desc);
        a.xy = reinterpret_cast<const float2 *>(views[k]->xy);
        a.angle = views[k]->angle;
        a.node = views[k]->node;
        a.level = views[k]->level;
        a.cell_w_inv = cc.cell_w_inv;
        a.cell_h_inv = cc.cell_h_inv;
        if ((e = launch_ingest(a, s))) return cuda_fail(e, "ingest kernel");
    }
    SearchConst sc;
    sc.hamming_max = sp.hamming_max;
    sc.ratio_num = sp.ratio_num;
    sc.ratio_den = sp.ratio_den;
    sc.epi_chi2 = sp.epi_chi2;
    sc.epipolar = sp.epipolar;
    sc.resolve = sp.resolve;
    sc.rot_filter = sp.rot_filter;
    sc.dense_min = 0;
    sc.epipole_px = sp.epipole_px;
    sc.rot_mode = sp.rot_mode;
    sc.baseline_min_ratio = 0.0f;  // (no median scene depth here)
    uint32_t *pair_offset = ps.running + 1;  // start of the output (always 0 here)
    if ((e = launch_pair_plain(slot_q, slot_t, q_free, t_free, q->n, t->n, kNoAllocMaxKp, sc, cc, ps,
                               reinterpret_cast<Out3 *>(out), pair_offset, ncmp, l, s)))
        return cuda_fail(e, "pair kernels");
    if ((e = cudaMemcpyAsync(n_out, ps.running, 4, cudaMemcpyDeviceToDevice, s))) return cuda_fail(e, "count");
    if (n_comparisons && (e = cudaMemcpyAsync(n_comparisons, ncmp, 8, cudaMemcpyDeviceToDevice, s)))
        return cuda_fail(e, "comparisons");
    return TM_OK;
}
