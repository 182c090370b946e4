// Host runtime of the C ABI (include/tm.h): context, keyframe store, batches, plans,
// autotuner.  The serving loop is in server.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "runtime.h"

#include <unordered_set>

namespace tmap {

// ------------------------------------------------------------------------- errors

static thread_local std::string g_error;

tm_status fail(tm_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

tm_status cuda_fail(cudaError_t e, const char *what) {
    return fail(TM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------------- buffers

cudaError_t DevBuf::reserve(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    release();
    size_t want = std::max<size_t>(256, n + n / 4);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) { p = nullptr; cap = 0; return e; }
    cap = want;
    ++generation;
    return cudaSuccess;
}
void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

cudaError_t PinBuf::reserve(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    release();
    size_t want = std::max<size_t>(4096, n + n / 4);
    cudaError_t e = cudaMallocHost(&p, want);
    if (e != cudaSuccess) { p = nullptr; cap = 0; return e; }
    cap = want;
    return cudaSuccess;
}
void PinBuf::release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (cudaHostAlloc / cudaHostRegister), which kernels
// may read directly; null for anything else.
const void *pinned_device_ptr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace tmap

using namespace tmap;

// ------------------------------------------------------------------------- context

extern "C" const char *tm_last_error(void) { return g_error.c_str(); }

extern "C" void tm_search_params_default(tm_search_params *p) {
    if (!p) return;
    p->hamming_max = 50;
    p->ratio_num = 3;
    p->ratio_den = 5;
    p->epi_chi2 = 3.84f;
    p->epipolar = 1;
    p->resolve = 1;
    p->rot_filter = 1;
    p->mode = TM_MODE_FUSED;
    p->lanes_per_query = 0;
    p->dense_min = 0;
    p->epipole_px = 0.0f;
    p->rot_mode = 0;
    p->baseline_min_ratio = 0.0f;
}

extern "C" void tm_triangulation_params_default(tm_triangulation_params *p) {
    if (!p) return;
    p->cos_parallax_max = 0.9998;
    p->chi2 = 5.991;
    p->ratio_factor = 1.5 * 1.2;
}

extern "C" void tm_fuse_params_default(tm_fuse_params *p) {
    if (!p) return;
    p->chi2 = 5.99f;
    p->hamming_max = 50;
    p->radius_scale = 3.0f;
}

extern "C" tm_status tm_ctx_create(int device, const tm_camera *cam, int32_t max_kp,
                                   size_t mem_budget_bytes, tm_ctx **out) {
    if (!out || !cam) return fail(TM_ERR_INVALID_ARG, "tm_ctx_create: null argument");
    *out = nullptr;
    if (max_kp < 1 || max_kp > TM_MAX_KP_LIMIT)
        return fail(TM_ERR_INVALID_ARG, "tm_ctx_create: max_kp %d outside [1, %d]", max_kp,
                    TM_MAX_KP_LIMIT);
    if (cam->width <= 0 || cam->height <= 0 || cam->width > TM_MAX_IMAGE_SIZE ||
        cam->height > TM_MAX_IMAGE_SIZE || !(cam->fx > 0) || !(cam->fy > 0))
        return fail(TM_ERR_INVALID_ARG, "tm_ctx_create: bad camera (image sides 1..%d px, fx, fy > 0)",
                    TM_MAX_IMAGE_SIZE);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(TM_ERR_INVALID_ARG, "tm_ctx_create: no device %d", device);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    tm_ctx *c = new tm_ctx();
    c->device = device;
    c->cam = *cam;
    c->cap = (max_kp + 31) & ~31;
    c->layout = SlotLayout::make(c->cap);
    c->slot_bytes = c->layout.bytes;
    c->budget = mem_budget_bytes;
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) { delete c; return cuda_fail(e, "props"); }
    c->num_sms = prop.multiProcessorCount;
    c->max_smem = prop.sharedMemPerBlockOptin;
    c->camc = CamConst::make(cam->fx, cam->fy, cam->cx, cam->cy, cam->width, cam->height);
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    const char *tc = getenv("TM_TUNE_CACHE");
    if (tc) load_tuning(c, tc);
    *out = c;
    return TM_OK;
}

tm_ctx::~tm_ctx() {
    cudaSetDevice(device);
    if (stream) cudaStreamSynchronize(stream);
    for (AsyncBatch &a : async) {
        if (a.s) cudaStreamSynchronize(a.s);
        if (a.B.mcopy) cudaStreamSynchronize(a.B.mcopy);
        a.B.release();
        if (a.ingested) cudaEventDestroy(a.ingested);
        if (a.s) cudaStreamDestroy(a.s);
    }
    batch.release();
    for (void *p : chunks) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
    if (capture_stream) cudaStreamDestroy(capture_stream);
}

extern "C" tm_status tm_ctx_destroy(tm_ctx *c) {
    if (!c) return fail(TM_ERR_INVALID_ARG, "tm_ctx_destroy: null");
    delete c;
    return TM_OK;
}

cudaStream_t tmap::pick_stream(tm_ctx *c, void *s) {
    return s ? static_cast<cudaStream_t>(s) : c->stream;
}

// ------------------------------------------------------------------------- store

tm_status tmap::alloc_slots_locked(tm_ctx *c, int n, std::vector<int> &got) {
    got.clear();
    while ((int)got.size() < n) {
        if (!c->free_slots.empty()) {
            got.push_back(c->free_slots.back());
            c->free_slots.pop_back();
            continue;
        }
        size_t max_slots = c->budget ? c->budget / c->slot_bytes : (size_t)-1;
        size_t have = c->slots.size();
        if (have >= max_slots) break;
        // chunks grow with the store (32, then as many as are held, at most 1024 slots), so
        // that a growing store allocates device memory a few times, not every 32 keyframes
        size_t want = std::min<size_t>(std::min<size_t>(std::max<size_t>(32, have), 1024), max_slots - have);
        want = std::max<size_t>(want, std::min<size_t>((size_t)(n - (int)got.size()), max_slots - have));
        size_t bytes = want * c->slot_bytes;
        if (!c->budget) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || fr < bytes + (size_t(1) << 30)) break;
        }
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        c->chunks.push_back(p);
        for (size_t k = 0; k < want; ++k) {
            Slot s;
            s.ptr = static_cast<unsigned char *>(p) + k * c->slot_bytes;
            c->slots.push_back(s);
            c->free_slots.push_back((int)c->slots.size() - 1);
        }
        // hand out lowest slot ids first
        std::sort(c->free_slots.begin(), c->free_slots.end(), std::greater<int>());
    }
    if ((int)got.size() < n) {
        for (int s : got) c->free_slots.push_back(s);
        got.clear();
        return fail(TM_ERR_NO_MEMORY, "keyframe store full (%zu slots of %zu bytes, budget %zu)",
                    c->slots.size(), c->slot_bytes, c->budget);
    }
    return TM_OK;
}

// Stage keyframes (host or device arrays) into the ingest buffers on stream s.  Slots must
// already be reserved.  The caller synchronizes before the staging buffers are reused.
tm_status tmap::classify_packed(tm_ctx *c, const tm_keyframes_packed &p, int n, std::vector<tm_keyframe_view> &views,
                                PackedSource &src) {
    if (n > 0 && (!p.n || !p.Tcw)) return fail(TM_ERR_INVALID_ARG, "packed keyframes: null counts or poses");
    size_t total = 0;
    for (int k = 0; k < n; ++k) {
        if (p.n[k] < 0 || p.n[k] > c->cap)
            return fail(TM_ERR_INVALID_ARG, "packed keyframe %d has %d keypoints, capacity %d", k, p.n[k], c->cap);
        total += (size_t)p.n[k];
    }
    src = PackedSource{};
    src.total = total;
    const void *arr[5] = {p.desc, p.xy, p.angle, p.node, p.level};
    if (total) {
        for (int q = 0; q < 5; ++q) {
            if (!arr[q]) return fail(TM_ERR_INVALID_ARG, "packed keyframes: null keypoint array");
            cudaPointerAttributes at;
            int kind = 3;
            const void *dp = arr[q];
            if (cudaPointerGetAttributes(&at, arr[q]) != cudaSuccess) {
                cudaGetLastError();
            } else if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
                if (at.type == cudaMemoryTypeDevice && at.device != c->device)
                    return fail(TM_ERR_INVALID_ARG, "packed keyframes: array on device %d, context on %d", at.device, c->device);
                kind = 1;
            } else if (at.type == cudaMemoryTypeHost && at.devicePointer) {
                kind = 2;
                dp = at.devicePointer;
            }
            if (q > 0 && kind != src.kind)
                return fail(TM_ERR_INVALID_ARG, "packed keyframes: arrays in different kinds of memory");
            src.kind = kind;
            src.src[q] = static_cast<const unsigned char *>(dp);
        }
        if (src.kind != 1) {
            // levels 0..7 use the low three bits only (one pass over all keyframes' levels)
            uint64_t any = 0;
            size_t i = 0;
            for (; i + 8 <= total; i += 8) {
                uint64_t w;
                memcpy(&w, p.level + i, 8);
                any |= w;
            }
            for (; i < total; ++i) any |= p.level[i];
            if (any & 0xF8F8F8F8F8F8F8F8ull)
                for (i = 0; i < total; ++i)
                    if (p.level[i] >= TM_LEVELS)
                        return fail(TM_ERR_INVALID_ARG, "packed keypoint %zu has level %d >= %d", i, p.level[i], TM_LEVELS);
        }
    }
    views.resize((size_t)n);
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        tm_keyframe_view &v = views[k];
        v.n = p.n[k];
        const bool any = v.n > 0;
        v.desc = any ? p.desc + 32 * off : nullptr;
        v.xy = any ? p.xy + 2 * off : nullptr;
        v.angle = any ? p.angle + off : nullptr;
        v.level = any ? p.level + off : nullptr;
        v.node = any ? p.node + off : nullptr;
        memcpy(v.Tcw, p.Tcw + 12 * (size_t)k, sizeof v.Tcw);
        off += (size_t)v.n;
    }
    return TM_OK;
}

tm_status tmap::stage_ingest(tm_ctx *c, IngestStage &st, int n, const tm_keyframe_view *kfs,
                             const int *slots, cudaStream_t s, IngestArgs &a, const PackedSource *pk) {
    size_t total = 0;
    for (int k = 0; k < n; ++k) total += (size_t)kfs[k].n;
    const size_t N = (total + 31) & ~size_t(31);
    // staged layout: desc | xy | angle | node | level | jobs
    const size_t o_desc = 0, o_xy = o_desc + N * 32, o_ang = o_xy + N * 8, o_node = o_ang + N * 4,
                 o_lvl = o_node + N * 4, o_jobs = align128(o_lvl + N),
                 bytes = align128(o_jobs + sizeof(IngestJob) * (size_t)n) + sizeof(GatherJob) * (size_t)n;
    cudaError_t e;
    if ((e = st.dev.reserve(bytes)) != cudaSuccess) return cuda_fail(e, "ingest staging");
    if ((e = st.host.reserve(bytes)) != cudaSuccess) return cuda_fail(e, "ingest pinned staging");
    unsigned char *h = static_cast<unsigned char *>(st.host.p);
    unsigned char *d = static_cast<unsigned char *>(st.dev.p);
    IngestJob *jobs = reinterpret_cast<IngestJob *>(h + o_jobs);
    size_t off = 0;
    st.src.assign((size_t)n, 0u);
    std::vector<GatherJob> gather;  // keyframes in page-locked host memory: read by a kernel
    for (int k = 0; k < n; ++k) {
        const tm_keyframe_view &v = kfs[k];
        const size_t m = (size_t)v.n;
        jobs[k].slot = c->slots[slots[k]].ptr;
        jobs[k].src = (uint32_t)off;
        st.src[k] = (uint32_t)off;
        jobs[k].n = v.n;
        for (int q = 0; q < 12; ++q) jobs[k].Tcw[q] = v.Tcw[q];
        if (pk) {  // packed: the arrays move once for all keyframes, below
            off += m;
            continue;
        }
        const void *pd[5] = {pinned_device_ptr(v.desc), pinned_device_ptr(v.xy), pinned_device_ptr(v.angle),
                             pinned_device_ptr(v.node), pinned_device_ptr(v.level)};
        if (m && pd[0] && pd[1] && pd[2] && pd[3] && pd[4]) {
            GatherJob g;
            for (int q = 0; q < 5; ++q) g.src[q] = static_cast<const unsigned char *>(pd[q]);
            g.dst = (uint32_t)off;
            g.n = (uint32_t)m;
            gather.push_back(g);
        } else if (m) {
            if (is_device_ptr(v.desc)) {
                if ((e = cudaMemcpyAsync(d + o_desc + off * 32, v.desc, m * 32, cudaMemcpyDeviceToDevice, s)) ||
                    (e = cudaMemcpyAsync(d + o_xy + off * 8, v.xy, m * 8, cudaMemcpyDeviceToDevice, s)) ||
                    (e = cudaMemcpyAsync(d + o_ang + off * 4, v.angle, m * 4, cudaMemcpyDeviceToDevice, s)) ||
                    (e = cudaMemcpyAsync(d + o_node + off * 4, v.node, m * 4, cudaMemcpyDeviceToDevice, s)) ||
                    (e = cudaMemcpyAsync(d + o_lvl + off, v.level, m, cudaMemcpyDeviceToDevice, s)))
                    return cuda_fail(e, "ingest copy");
            } else {
                memcpy(h + o_desc + off * 32, v.desc, m * 32);
                memcpy(h + o_xy + off * 8, v.xy, m * 8);
                memcpy(h + o_ang + off * 4, v.angle, m * 4);
                memcpy(h + o_node + off * 4, v.node, m * 4);
                memcpy(h + o_lvl + off, v.level, m);
                st.host_ranges.push_back({off, m});
            }
        }
        off += m;
    }
    if (pk && pk->total) {
        // the packed arrays are laid out as the staging area is (keyframes in order)
        const size_t T = pk->total;
        const size_t o5[5] = {o_desc, o_xy, o_ang, o_node, o_lvl}, e5[5] = {32, 8, 4, 4, 1};
        if (pk->kind == 1) {
            for (int q = 0; q < 5; ++q)
                if ((e = cudaMemcpyAsync(d + o5[q], pk->src[q], T * e5[q], cudaMemcpyDeviceToDevice, s)))
                    return cuda_fail(e, "ingest copy");
        } else if (pk->kind == 2) {
            // page-locked: read by the gather kernel in chunks of 1024 keypoints
            constexpr size_t kChunk = 1024;
            for (size_t o = 0; o < T; o += kChunk) {
                GatherJob g;
                for (int q = 0; q < 5; ++q) g.src[q] = pk->src[q] + o * e5[q];
                g.dst = (uint32_t)o;
                g.n = (uint32_t)std::min(kChunk, T - o);
                gather.push_back(g);
            }
        } else {
            for (int q = 0; q < 5; ++q) memcpy(h + o5[q], pk->src[q], T * e5[q]);
            st.host_ranges.push_back({0, T});
        }
    }
    // one transfer of everything staged on the host (contiguous runs merged per array)
    auto flush = [&](size_t base, size_t elt) -> cudaError_t {
        size_t a = 0;
        while (a < st.host_ranges.size()) {
            size_t b = a;
            size_t lo = st.host_ranges[a].first, hi = lo + st.host_ranges[a].second;
            while (b + 1 < st.host_ranges.size() && st.host_ranges[b + 1].first == hi) {
                ++b;
                hi += st.host_ranges[b].second;
            }
            cudaError_t r = cudaMemcpyAsync(d + base + lo * elt, h + base + lo * elt, (hi - lo) * elt,
                                            cudaMemcpyHostToDevice, s);
            if (r != cudaSuccess) return r;
            a = b + 1;
        }
        return cudaSuccess;
    };
    if ((e = flush(o_desc, 32)) || (e = flush(o_xy, 8)) || (e = flush(o_ang, 4)) ||
        (e = flush(o_node, 4)) || (e = flush(o_lvl, 1)))
        return cuda_fail(e, "ingest upload");
    st.host_ranges.clear();
    if ((e = cudaMemcpyAsync(d + o_jobs, jobs, sizeof(IngestJob) * (size_t)n, cudaMemcpyHostToDevice, s)))
        return cuda_fail(e, "ingest jobs upload");
    if (!gather.empty()) {
        // the gather jobs follow the ingest jobs in both staging areas
        const size_t o_g = align128(o_jobs + sizeof(IngestJob) * (size_t)n);
        const size_t gb = sizeof(GatherJob) * gather.size();
        if (o_g + gb > st.dev.cap || o_g + gb > st.host.cap) return fail(TM_ERR_CUDA, "ingest staging: gather jobs");
        memcpy(h + o_g, gather.data(), gb);
        const size_t offs[5] = {o_desc, o_xy, o_ang, o_node, o_lvl};
        if ((e = cudaMemcpyAsync(d + o_g, h + o_g, gb, cudaMemcpyHostToDevice, s)) ||
            (e = launch_stage_gather(reinterpret_cast<const GatherJob *>(d + o_g), (int)gather.size(), d, offs, s)))
            return cuda_fail(e, "ingest staging gather");
    }
    a.jobs = reinterpret_cast<const IngestJob *>(d + o_jobs);
    a.n_jobs = n;
    a.cap = c->cap;
    a.desc = reinterpret_cast<const uint4 *>(d + o_desc);
    a.xy = reinterpret_cast<const float2 *>(d + o_xy);
    a.angle = reinterpret_cast<const float *>(d + o_ang);
    a.node = reinterpret_cast<const uint32_t *>(d + o_node);
    a.level = d + o_lvl;
    a.cell_w_inv = c->camc.cell_w_inv;
    a.cell_h_inv = c->camc.cell_h_inv;
    return TM_OK;
}

tm_status tmap::enqueue_ingest(tm_ctx *c, IngestStage &st, int n, const tm_keyframe_view *kfs,
                               const int *slots, cudaStream_t s) {
    IngestArgs a;
    tm_status r = stage_ingest(c, st, n, kfs, slots, s, a);
    if (r) return r;
    cudaError_t e = launch_ingest(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "ingest kernel");
    return TM_OK;
}

tm_status tmap::validate_view(tm_ctx *c, const tm_keyframe_view &v) {
    if (v.n < 0 || v.n > c->cap)
        return fail(TM_ERR_INVALID_ARG, "keyframe has %d keypoints, capacity %d", v.n, c->cap);
    if (v.n > 0 && (!v.desc || !v.xy || !v.angle || !v.level || !v.node))
        return fail(TM_ERR_INVALID_ARG, "keyframe arrays must be non-null");
    if (v.n > 0 && !is_device_ptr(v.level)) {
        // levels 0..7 use the low three bits only: or the bytes together 8 at a time, and
        // look for the offending keypoint only if some byte has a higher bit set
        static_assert(TM_LEVELS == 8, "the level check assumes 8 levels");
        uint64_t any = 0;
        int i = 0;
        for (; i + 8 <= v.n; i += 8) {
            uint64_t w;
            memcpy(&w, v.level + i, 8);
            any |= w;
        }
        for (; i < v.n; ++i) any |= v.level[i];
        if (any & 0xF8F8F8F8F8F8F8F8ull)
            for (i = 0; i < v.n; ++i)
                if (v.level[i] >= TM_LEVELS)
                    return fail(TM_ERR_INVALID_ARG, "keypoint %d has level %d >= %d", i, v.level[i], TM_LEVELS);
    }
    return TM_OK;
}

tm_status tmap::store_add(tm_ctx *c, int n, const uint64_t *ids, const tm_keyframe_view *kfs,
                        cudaStream_t s, std::vector<int> &slots) {
    for (int k = 0; k < n; ++k) {
        tm_status st = validate_view(c, kfs[k]);
        if (st) return st;
        if (c->ids.count(ids[k])) return fail(TM_ERR_EXISTS, "keyframe %llu already stored", (unsigned long long)ids[k]);
        for (int q = 0; q < k; ++q)
            if (ids[q] == ids[k]) return fail(TM_ERR_EXISTS, "keyframe %llu given twice", (unsigned long long)ids[k]);
    }
    tm_status st = alloc_slots_locked(c, n, slots);
    if (st) return st;
    st = enqueue_ingest(c, c->ingest, n, kfs, slots.data(), s);
    if (st) {
        for (int sl : slots) c->free_slots.push_back(sl);
        return st;
    }
    for (int k = 0; k < n; ++k) {
        c->slots[slots[k]].n = kfs[k].n;
        c->slots[slots[k]].refs = 0;
        c->slots[slots[k]].id = ids[k];
        c->ids[ids[k]] = slots[k];
    }
    return TM_OK;
}

extern "C" tm_status tm_store_add_keyframes(tm_ctx *c, int32_t n, const uint64_t *ids,
                                            const tm_keyframe_view *kfs, void *stream) {
    if (!c || n < 0 || (n > 0 && (!ids || !kfs))) return fail(TM_ERR_INVALID_ARG, "tm_store_add_keyframes: bad arguments");
    if (n == 0) return TM_OK;
    Range range("tm_store_add_keyframes");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaStream_t s = pick_stream(c, stream);
    std::vector<int> slots;
    tm_status st = store_add(c, n, ids, kfs, s, slots);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ingest");
    return TM_OK;
}

extern "C" tm_status tm_store_reserve(tm_ctx *c, int32_t n_slots) {
    if (!c || n_slots < 0) return fail(TM_ERR_INVALID_ARG, "tm_store_reserve: bad arguments");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    const size_t free_now = c->free_slots.size();
    if ((size_t)n_slots <= free_now) return TM_OK;
    // allocate the missing slots in one chunk (within the budget), keeping them free
    const size_t max_slots = c->budget ? c->budget / c->slot_bytes : (size_t)-1;
    const size_t want = std::min<size_t>((size_t)n_slots - free_now, max_slots - std::min(max_slots, c->slots.size()));
    if (want == 0) return fail(TM_ERR_NO_MEMORY, "tm_store_reserve: budget holds %zu slots", c->slots.size());
    if (!c->budget) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || fr < want * c->slot_bytes + (size_t(1) << 30))
            return fail(TM_ERR_NO_MEMORY, "tm_store_reserve: not enough free device memory");
    }
    void *p = nullptr;
    if (cudaMalloc(&p, want * c->slot_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(TM_ERR_NO_MEMORY, "tm_store_reserve: allocation of %zu slots failed", want);
    }
    c->chunks.push_back(p);
    for (size_t k = 0; k < want; ++k) {
        Slot sl;
        sl.ptr = static_cast<unsigned char *>(p) + k * c->slot_bytes;
        c->slots.push_back(sl);
        c->free_slots.push_back((int)c->slots.size() - 1);
    }
    std::sort(c->free_slots.begin(), c->free_slots.end(), std::greater<int>());
    return (size_t)n_slots <= c->free_slots.size() ? TM_OK
                                                   : fail(TM_ERR_NO_MEMORY, "tm_store_reserve: budget reached");
}

extern "C" tm_status tm_store_add_keyframe(tm_ctx *c, uint64_t id, const tm_keyframe_view *kf,
                                           void *stream) {
    return tm_store_add_keyframes(c, 1, &id, kf, stream);
}

extern "C" tm_status tm_store_remove_keyframe(tm_ctx *c, uint64_t id) {
    if (!c) return fail(TM_ERR_INVALID_ARG, "null context");
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->ids.find(id);
    if (it == c->ids.end()) return fail(TM_ERR_NOT_FOUND, "keyframe %llu not stored", (unsigned long long)id);
    Slot &sl = c->slots[it->second];
    if (sl.refs > 0) return fail(TM_ERR_BUSY, "keyframe %llu is used by %d live plan(s)", (unsigned long long)id, sl.refs);
    sl.n = 0;
    c->free_slots.push_back(it->second);
    c->ids.erase(it);
    return TM_OK;
}

extern "C" tm_status tm_store_remove_keyframes(tm_ctx *c, int32_t n, const uint64_t *ids) {
    if (!c || n < 0 || (n > 0 && !ids)) return fail(TM_ERR_INVALID_ARG, "tm_store_remove_keyframes: bad arguments");
    std::lock_guard<std::mutex> lk(c->mu);
    // all or nothing: every id is checked before any slot is freed
    std::unordered_set<uint64_t> seen;
    seen.reserve((size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        auto it = c->ids.find(ids[k]);
        if (it == c->ids.end()) return fail(TM_ERR_NOT_FOUND, "keyframe %llu not stored", (unsigned long long)ids[k]);
        const Slot &sl = c->slots[it->second];
        if (sl.refs > 0)
            return fail(TM_ERR_BUSY, "keyframe %llu is used by %d live plan(s)", (unsigned long long)ids[k], sl.refs);
        if (!seen.insert(ids[k]).second)
            return fail(TM_ERR_INVALID_ARG, "keyframe %llu given twice", (unsigned long long)ids[k]);
    }
    for (int32_t k = 0; k < n; ++k) {
        auto it = c->ids.find(ids[k]);
        c->slots[it->second].n = 0;
        c->free_slots.push_back(it->second);
        c->ids.erase(it);
    }
    return TM_OK;
}

extern "C" tm_status tm_store_keyframe_size(tm_ctx *c, uint64_t id, int32_t *n) {
    if (!c || !n) return fail(TM_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->ids.find(id);
    if (it == c->ids.end()) return fail(TM_ERR_NOT_FOUND, "keyframe %llu not stored", (unsigned long long)id);
    *n = c->slots[it->second].n;
    return TM_OK;
}

extern "C" tm_status tm_store_get_stats(tm_ctx *c, tm_store_stats *o) {
    if (!c || !o) return fail(TM_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    o->device = c->device;
    o->max_kp = c->cap;
    o->slots_used = (int)c->ids.size();
    size_t max_slots = c->budget ? c->budget / c->slot_bytes : 0;
    o->slots_free_in_budget = c->budget ? (int)(max_slots - c->ids.size()) : -1;
    o->slot_bytes = c->slot_bytes;
    o->bytes_reserved = c->slots.size() * c->slot_bytes;
    o->budget_bytes = c->budget;
    return TM_OK;
}

// ------------------------------------------------------------------------- batches

void BatchBuf::release() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_timed) cudaGraphExecDestroy(graph_timed);
    graph = graph_timed = nullptr;
    for (DevBuf *b : {&items, &masks, &mp_pos, &mp_normal, &mp_desc, &mp_min, &mp_max,
                      &mp_skip, &padded, &counts, &item_cmp, &offsets, &ncmp, &counters, &dense, &scratch, &dres, &acc, &pconst, &pwords, &pepos, &work, &points, &point_ok, &pwin, &pacc, &pdone, &ents, &povf, &mp_block})
        b->release();
    h_stage.release();
    h_out.release();
    ingest.release();
    for (cudaEvent_t &e : ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (pfork) cudaEventDestroy(pfork);
    if (paux) cudaStreamDestroy(paux);
    if (join) cudaEventDestroy(join);
    pfork = join = nullptr;
    paux = nullptr;
    if (mpre) cudaEventDestroy(mpre);
    if (mready) cudaEventDestroy(mready);
    if (mcopy) cudaStreamDestroy(mcopy);
    mpre = mready = nullptr;
    mcopy = nullptr;
    forked = mp_async = false;
}

// The search branch's stream and events, and the map-point copy stream, created on first use.
static tm_status ensure_branches(BatchBuf &B) {
    cudaError_t e;
    if (!B.paux && ((e = cudaStreamCreateWithFlags(&B.paux, cudaStreamNonBlocking)) ||
                    (e = cudaEventCreateWithFlags(&B.pfork, cudaEventDisableTiming)) ||
                    (e = cudaEventCreateWithFlags(&B.join, cudaEventDisableTiming))))
        return cuda_fail(e, "launch branches");
    if (!B.mcopy && ((e = cudaStreamCreateWithFlags(&B.mcopy, cudaStreamNonBlocking)) ||
                     (e = cudaEventCreateWithFlags(&B.mpre, cudaEventDisableTiming)) ||
                     (e = cudaEventCreateWithFlags(&B.mready, cudaEventDisableTiming))))
        return cuda_fail(e, "map point stream");
    return TM_OK;
}

static SearchConst to_const(const tm_search_params &p) {
    SearchConst s;
    s.hamming_max = p.hamming_max;
    s.ratio_num = p.ratio_num;
    s.ratio_den = p.ratio_den;
    s.epi_chi2 = p.epi_chi2;
    s.epipolar = p.epipolar;
    s.resolve = p.resolve;
    s.rot_filter = p.rot_filter;
    s.dense_min = p.mode == TM_MODE_FUSED ? p.dense_min : 0;
    s.epipole_px = p.epipole_px;
    s.rot_mode = p.rot_mode;
    s.baseline_min_ratio = p.baseline_min_ratio;
    return s;
}

static tm_status check_params(const tm_search_params &sp, const tm_fuse_params &fp) {
    if (sp.hamming_max < 0 || sp.ratio_num < 0 || sp.ratio_den < 0 || !(sp.epi_chi2 >= 0))
        return fail(TM_ERR_INVALID_ARG, "bad search parameters");
    if (sp.mode != TM_MODE_FUSED && sp.mode != TM_MODE_PER_PAIR)
        return fail(TM_ERR_INVALID_ARG, "bad search mode %d", sp.mode);
    if (sp.dense_min != 0 && sp.dense_min != -1 && sp.dense_min < 16)
        return fail(TM_ERR_INVALID_ARG, "dense_min must be 0, -1 (tuned) or >= 16 (got %d)", sp.dense_min);
    if (!(sp.epipole_px >= 0.0f && sp.epipole_px < 1e6f))
        return fail(TM_ERR_INVALID_ARG, "epipole_px must be in [0, 1e6)");
    if (sp.rot_mode != 0 && sp.rot_mode != 1) return fail(TM_ERR_INVALID_ARG, "rot_mode must be 0 or 1");
    if (!(sp.baseline_min_ratio >= 0.0f && sp.baseline_min_ratio < 1e6f))
        return fail(TM_ERR_INVALID_ARG, "baseline_min_ratio must be in [0, 1e6)");
    const int l = sp.lanes_per_query;
    if (!(l == 0 || l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32))
        return fail(TM_ERR_INVALID_ARG, "lanes_per_query must be 0, 1, 2, 4, 8, 16 or 32");
    if (fp.hamming_max < 0 || !(fp.chi2 >= 0) || !(fp.radius_scale >= 0))
        return fail(TM_ERR_INVALID_ARG, "bad fuse parameters");
    return TM_OK;
}

// Build the work list of a batch and upload everything it needs (one transfer per array).
// Caller holds c->mu.  On success B describes the batch and its slots are listed in B.slots.
tm_status tmap::prepare_batch(tm_ctx *c, BatchBuf &B, const tm_step *steps, int n_steps,
                            const tm_batch_inputs *in, const tm_search_params &sp,
                            const tm_fuse_params &fp, cudaStream_t s) {
    tm_status st = check_params(sp, fp);
    if (st) return st;
    if (n_steps < 0 || (n_steps > 0 && !steps)) return fail(TM_ERR_INVALID_ARG, "bad steps");
    const size_t mask_bytes = in ? in->mask_bytes : 0;
    const tm_mappoint_view mps = in ? in->mps : tm_mappoint_view{};
    const tm_triangulation_params *tri = in ? in->tri : nullptr;
    if (tri && !(tri->cos_parallax_max > 0.0 && tri->cos_parallax_max <= 1.0 && tri->chi2 >= 0.0 &&
                 tri->ratio_factor >= 1.0))
        return fail(TM_ERR_INVALID_ARG, "bad triangulation parameters");
    if (mask_bytes && !in->masks) return fail(TM_ERR_INVALID_ARG, "masks is null");
    if (mps.n < 0) return fail(TM_ERR_INVALID_ARG, "negative map point count");
    if (mps.n > 0 && (!mps.pos || !mps.normal || !mps.desc || !mps.min_dist || !mps.max_dist))
        return fail(TM_ERR_INVALID_ARG, "map point arrays must be non-null");
    std::vector<void *> before = B.pointers();
    // map points in one caller block: the byte offset of each array in it (checked: inside the
    // block, aligned as the kernels read it), so that the block is uploaded with one copy
    const unsigned char *blk = in ? static_cast<const unsigned char *>(in->mps_block) : nullptr;
    const uint64_t blk_bytes = in ? in->mps_block_bytes : 0;
    uint64_t boff[6] = {0, 0, 0, 0, 0, 0};  // pos, normal, desc, min_dist, max_dist, skip
    if (blk && mps.n > 0) {
        const size_t m = (size_t)mps.n;
        const void *ptr[6] = {mps.pos, mps.normal, mps.desc, mps.min_dist, mps.max_dist, mps.skip};
        const size_t len[6] = {m * 12, m * 12, m * 32, m * 4, m * 4, m};
        const unsigned align[6] = {4, 4, 16, 4, 4, 1};
        for (int k = 0; k < 6; ++k) {
            if (!ptr[k]) continue;
            const unsigned char *p = static_cast<const unsigned char *>(ptr[k]);
            if (p < blk || (uint64_t)(p - blk) > blk_bytes || len[k] > blk_bytes - (uint64_t)(p - blk) ||
                (uint64_t)(p - blk) % align[k])
                return fail(TM_ERR_INVALID_ARG, "map point array %d outside the block or off alignment", k);
            boff[k] = (uint64_t)(p - blk);
        }
    } else {
        blk = nullptr;
    }
    // the map points' upload: the block with one copy, or the six arrays
    auto upload_mps = [&](cudaStream_t cs) -> cudaError_t {
        const size_t m = (size_t)mps.n;
        cudaError_t ce;
        if (blk) {
            if ((ce = B.mp_block.reserve(std::max<uint64_t>(16, blk_bytes)))) return ce;
            return cudaMemcpyAsync(B.mp_block.p, blk, blk_bytes, cudaMemcpyDefault, cs);
        }
        if ((ce = cudaMemcpyAsync(B.mp_pos.p, mps.pos, m * 12, cudaMemcpyDefault, cs)) ||
            (ce = cudaMemcpyAsync(B.mp_normal.p, mps.normal, m * 12, cudaMemcpyDefault, cs)) ||
            (ce = cudaMemcpyAsync(B.mp_desc.p, mps.desc, m * 32, cudaMemcpyDefault, cs)) ||
            (ce = cudaMemcpyAsync(B.mp_min.p, mps.min_dist, m * 4, cudaMemcpyDefault, cs)) ||
            (ce = cudaMemcpyAsync(B.mp_max.p, mps.max_dist, m * 4, cudaMemcpyDefault, cs)))
            return ce;
        return mps.skip ? cudaMemcpyAsync(B.mp_skip.p, mps.skip, m, cudaMemcpyDefault, cs) : cudaSuccess;
    };
    // a one-shot batch copies its map points first, on a stream of their own that only the
    // fusion kernel awaits, so that the copy runs under the host work below
    B.forked = B.mp_async = false;
    bool mp_copied = false;
    if (B.early_fork && mps.n > 0) {
        const size_t m = (size_t)mps.n;
        cudaError_t e;
        if ((st = ensure_branches(B))) return st;
        if ((e = B.mp_pos.reserve(m * 12)) || (e = B.mp_normal.reserve(m * 12)) || (e = B.mp_desc.reserve(m * 32)) ||
            (e = B.mp_min.reserve(m * 4)) || (e = B.mp_max.reserve(m * 4)) || (e = B.mp_skip.reserve(m)))
            return cuda_fail(e, "batch buffers");
        if ((e = cudaEventRecord(B.mpre, s)) || (e = cudaStreamWaitEvent(B.mcopy, B.mpre, 0)))
            return cuda_fail(e, "map point stream");
        if ((e = upload_mps(B.mcopy)) || (e = cudaEventRecord(B.mready, B.mcopy)))
            return cuda_fail(e, "map point upload");
        B.mp_async = mp_copied = true;
    }
    // keyframes entering the store with this batch: reserve slots and stage them; the ingest
    // kernel runs at the head of every launch of the batch
    B.n_new = 0;
    std::vector<int> new_slots;
    const int n_new = in ? in->n_new : 0;
    if (n_new < 0 || (n_new > 0 && (!in->new_ids || (!in->new_kfs && !in->new_packed))))
        return fail(TM_ERR_INVALID_ARG, "bad new keyframes");
    std::vector<tm_keyframe_view> packed_views;
    PackedSource packed_src;
    const bool packed = n_new > 0 && !in->new_kfs;
    if (packed && (st = classify_packed(c, *in->new_packed, n_new, packed_views, packed_src))) return st;
    const tm_keyframe_view *new_kfs = packed ? packed_views.data() : (in ? in->new_kfs : nullptr);
    if (n_new > 0) {
        for (int k = 0; k < n_new; ++k) {
            if (!packed && (st = validate_view(c, new_kfs[k]))) return st;
            if (c->ids.count(in->new_ids[k]))
                return fail(TM_ERR_EXISTS, "keyframe %llu already stored", (unsigned long long)in->new_ids[k]);
            for (int q = 0; q < k; ++q)
                if (in->new_ids[q] == in->new_ids[k])
                    return fail(TM_ERR_EXISTS, "keyframe %llu given twice", (unsigned long long)in->new_ids[k]);
        }
        if ((st = alloc_slots_locked(c, n_new, new_slots))) return st;
        if ((st = stage_ingest(c, B.ingest, n_new, new_kfs, new_slots.data(), s, B.ingest_args,
                               packed ? &packed_src : nullptr))) {
            for (int sl : new_slots) c->free_slots.push_back(sl);
            return st;
        }
        for (int k = 0; k < n_new; ++k) {
            Slot &sl = c->slots[new_slots[k]];
            sl.n = new_kfs[k].n;
            sl.refs = 0;
            sl.id = in->new_ids[k];
            c->ids[in->new_ids[k]] = new_slots[k];
        }
        B.n_new = n_new;
    }
    // on failure below, the new keyframes are taken out of the store again
    struct Rollback {
        tm_ctx *c; const tm_batch_inputs *in; std::vector<int> *slots; BatchBuf *B; bool armed = true;
        ~Rollback() {
            if (!armed || slots->empty()) return;
            for (size_t k = 0; k < slots->size(); ++k) {
                c->ids.erase(in->new_ids[k]);
                c->free_slots.push_back((*slots)[k]);
            }
            B->n_new = 0;
        }
    } rollback{c, in, &new_slots, &B};
    // pose of a keyframe as the search kernel reads it: from the slot header, or from the
    // ingest job of a keyframe entering with this batch (so that the search need not wait for
    // its ingest)
    // slot -> position among the keyframes entering with this batch, -1 for stored ones
    std::vector<int> &new_index = B.new_index;
    new_index.assign(c->slots.size(), -1);
    for (size_t k = 0; k < new_slots.size(); ++k) new_index[(size_t)new_slots[k]] = (int)k;
    auto pose_of = [&](int slot) -> const double * {
        const int ni = new_index[(size_t)slot];
        const unsigned char *p = ni >= 0
            ? reinterpret_cast<const unsigned char *>(B.ingest_args.jobs) + sizeof(IngestJob) * (size_t)ni +
                  offsetof(IngestJob, Tcw)
            : c->slots[slot].ptr + offsetof(KfHeader, Tcw);
        return reinterpret_cast<const double *>(p);
    };
    // where the search reads a query keyframe: a stored one from its slot, one entering with
    // this batch from its staged caller-order arrays (so that the search need not wait for its
    // ingest)
    const SlotLayout SL = SlotLayout::make(c->cap);
    struct QView { const uint4 *desc; const float2 *xy; const uint32_t *node; const uint16_t *orig;
                   const float *angle; uint32_t raw; };
    auto qview_of = [&](int slot) -> QView {
        const int ni = new_index[(size_t)slot];
        if (ni >= 0) {
            const IngestArgs &a = B.ingest_args;
            const uint32_t src = B.ingest.src[(size_t)ni];
            return QView{a.desc + 2 * (size_t)src, a.xy + src, a.node + src, nullptr, a.angle + src, 1u};
        }
        const unsigned char *b = c->slots[slot].ptr;
        return QView{reinterpret_cast<const uint4 *>(b + SL.desc), reinterpret_cast<const float2 *>(b + SL.xy),
                     reinterpret_cast<const uint32_t *>(b + SL.node), reinterpret_cast<const uint16_t *>(b + SL.orig),
                     reinterpret_cast<const float *>(b + SL.angle), 0u};
    };
    B.nbr_new = false;
    std::vector<WorkItem> &items = B.h_items;

    items.clear();
    B.item_nq.clear();
    B.item_nt.clear();
    size_t n_pairs_max = 0;
    for (int k = 0; k < n_steps; ++k) n_pairs_max += (size_t)std::max(0, steps[k].n_nbrs);
    // split_min > 0: split in batches of fewer pairs than SMs; < 0: split whatever the batch.
    // Split pairs run the default gates (the epipole rejection and dense blocks: never split).
    const bool split = (c->split_min < 0 || (c->split_min > 0 && n_pairs_max < (size_t)c->num_sms)) &&
                       !(sp.epipole_px > 0.0f) && sp.dense_min == 0 && sp.mode != TM_MODE_PER_PAIR;
    items.reserve(n_pairs_max + 64);
    B.item_nq.reserve(n_pairs_max);
    B.item_nt.reserve(n_pairs_max);
    std::vector<int> slots_used;
    slots_used.reserve(n_pairs_max + (size_t)n_steps + new_slots.size());
    B.step_pair_begin.assign(n_steps + 1, 0);
    B.step_fuse_item.assign(n_steps + 1, 0);
    B.n_pairs = 0;
    uint32_t pad = 0, dq = 0, tq = 0;
    int smem_n = 32;
    auto slot_of = [&](uint64_t id, int &slot) -> tm_status {
        auto it = c->ids.find(id);
        if (it == c->ids.end()) return fail(TM_ERR_NOT_FOUND, "keyframe %llu not stored", (unsigned long long)id);
        slot = it->second;
        // a keyframe an asynchronous batch is still storing: only later asynchronous batches,
        // which wait for that ingest, may read it before the batch is finished
        if (c->slots[slot].pending && !B.allow_pending)
            return fail(TM_ERR_BUSY, "keyframe %llu is being stored by a batch in flight (tm_batch_finish it first)",
                        (unsigned long long)id);
        return TM_OK;
    };
    for (int k = 0; k < n_steps; ++k) {
        const tm_step &S = steps[k];
        int qs = -1;
        if ((st = slot_of(S.kf_id, qs))) return st;
        const int nq = c->slots[qs].n;
        if (S.n_nbrs < 0 || (S.n_nbrs > 0 && !S.nbr_ids)) return fail(TM_ERR_INVALID_ARG, "step %d: bad neighbours", k);
        if (S.q_free_off >= 0 && (size_t)S.q_free_off + (size_t)nq > mask_bytes)
            return fail(TM_ERR_INVALID_ARG, "step %d: query mask outside masks", k);
        B.step_pair_begin[k] = B.n_pairs;
        size_t toff = S.nbr_free_off >= 0 ? (size_t)S.nbr_free_off : 0;
        const double *pq = pose_of(qs);  // the query keyframe's parts, once per step
        const QView qv = qview_of(qs);
        unsigned char *qptr = c->slots[qs].ptr;
        for (int j = 0; j < S.n_nbrs; ++j) {
            int ts = -1;
            if ((st = slot_of(S.nbr_ids[j], ts))) return st;
            const int nt = c->slots[ts].n;
            if (S.nbr_free_off >= 0 && toff + (size_t)nt > mask_bytes)
                return fail(TM_ERR_INVALID_ARG, "step %d: neighbour masks outside masks", k);
            WorkItem w{};
            w.q = qptr;
            w.t = c->slots[ts].ptr;
            w.pq = pq;
            const bool t_new = new_index[(size_t)ts] >= 0;
            w.pt = pose_of(ts);
            w.mdepth = S.nbr_median_depth ? S.nbr_median_depth[j] : 0.0f;
            w.qdesc = qv.desc;
            w.qxy = qv.xy;
            w.qnode = qv.node;
            w.qorig = qv.orig;
            w.qangle = qv.angle;
            w.qraw = qv.raw;
            B.nbr_new |= t_new;
            w.kind = kItemSearch;
            // pairs with many queries are split over two search CTAs (part | parts << 8) when the
            // batch's pairs are fewer than the SMs (a full batch fills the GPU unsplit, and
            // there the split's second setup and global winners cost more than they gain)
            w.step = (split && nq >= std::abs(c->split_min)) ? 2u << 8 : 1u << 8;
            w.out_off = pad;
            w.a = S.q_free_off >= 0 ? (uint32_t)S.q_free_off : kNone;
            w.b = S.nbr_free_off >= 0 ? (uint32_t)toff : kNone;
            w.nq = (uint32_t)nq;
            w.nt = (uint32_t)nt;
            w.cost = (uint32_t)std::min<uint64_t>(0xFFFFFFFFull, (uint64_t)nq + nt + (uint64_t)nq * nt / 256);
            w.c = dq;
            dq += (uint32_t)nq;
            // per-target arrays of the prep kernel: the eligible positions and the bitmap words
            // (nwt + 1 of them) from toff / 32, a multiple of 64 (16-byte aligned copies)
            w.toff = tq;
            tq += (uint32_t)((32 * ((nt + 31) / 32 + 1) + 63) & ~63);
            pad += (uint32_t)(sp.resolve ? std::min(nq, nt) : nq);
            smem_n = std::max(smem_n, std::max(nq, nt));
            items.push_back(w);
            B.item_nq.push_back(nq);
            B.item_nt.push_back(nt);
            slots_used.push_back(ts);
            toff += (size_t)nt;
            ++B.n_pairs;
        }
        slots_used.push_back(qs);
    }
    B.step_pair_begin[n_steps] = B.n_pairs;
    B.n_search_items = (uint32_t)items.size();
    B.search_pad = pad;
    for (int k = 0; k < n_steps; ++k) {
        const tm_step &S = steps[k];
        B.step_fuse_item[k] = (int)items.size();
        if (S.mp_count <= 0) continue;
        if (S.mp_begin < 0 || (int64_t)S.mp_begin + S.mp_count > mps.n)
            return fail(TM_ERR_INVALID_ARG, "step %d: map point range outside the batch", k);
        const int qs = c->ids[S.kf_id];
        for (int b = 0; b < S.mp_count; b += kFuseChunk) {
            WorkItem w{};
            w.q = c->slots[qs].ptr;
            w.kind = kItemFuse;
            w.out_off = pad;
            w.a = (uint32_t)(S.mp_begin + b);
            w.b = (uint32_t)std::min(kFuseChunk, S.mp_count - b);
            w.c = (uint32_t)S.mp_begin;
            w.nt = (uint32_t)c->slots[qs].n;
            w.step = (uint32_t)k;
            w.skip = kNone;
            w.cost = 2 * w.b;
            pad += w.b;
            items.push_back(w);
        }
    }
    B.step_fuse_item[n_steps] = (int)items.size();
    B.n_bwd_items = (uint32_t)items.size() - B.n_search_items;
    // forward fusion: the new keyframe's map points into each neighbour (Sec. IV-D)
    B.pair_fwd_item.assign((size_t)B.n_pairs + 1, 0);
    B.any_fwd = false;
    {
        int p = 0;
        for (int k = 0; k < n_steps; ++k) {
            const tm_step &S = steps[k];
            const int cnt = S.fwd_mp_count;
            if (cnt < 0 || (cnt > 0 && (S.fwd_mp_begin < 0 || (int64_t)S.fwd_mp_begin + cnt > mps.n)))
                return fail(TM_ERR_INVALID_ARG, "step %d: forward map point range outside the batch", k);
            if (cnt > 0 && S.fwd_skip_off >= 0 &&
                (size_t)S.fwd_skip_off + (size_t)S.n_nbrs * (size_t)cnt > mask_bytes)
                return fail(TM_ERR_INVALID_ARG, "step %d: forward skip bytes outside masks", k);
            for (int j = 0; j < S.n_nbrs; ++j, ++p) {
                B.pair_fwd_item[p] = (int)items.size();
                if (cnt <= 0) continue;
                B.any_fwd = true;
                const int ts = c->ids[S.nbr_ids[j]];
                for (int b = 0; b < cnt; b += kFuseChunk) {
                    WorkItem w{};
                    w.q = c->slots[ts].ptr;
                    w.kind = kItemFuse;
                    w.out_off = pad;
                    w.a = (uint32_t)(S.fwd_mp_begin + b);
                    w.b = (uint32_t)std::min(kFuseChunk, cnt - b);
                    w.c = (uint32_t)S.fwd_mp_begin;
                    w.nt = (uint32_t)c->slots[ts].n;
                    w.step = (uint32_t)k;
                    w.skip = S.fwd_skip_off >= 0 ? (uint32_t)((size_t)S.fwd_skip_off + (size_t)j * cnt + b) : kNone;
                    w.cost = 2 * w.b;
                    pad += w.b;
                    items.push_back(w);
                }
            }
        }
        B.pair_fwd_item[B.n_pairs] = (int)items.size();
    }
    for (int sl : new_slots) slots_used.push_back(sl);
    B.n_items = (uint32_t)items.size();
    B.n_steps = n_steps;
    B.total_pad = pad;
    B.smem_n = (smem_n + 31) & ~31;
    B.slots = slots_used;
    // search CTAs take the pairs largest first (ties in item order): one 64-bit key per pair,
    // (~cost << 32 | index), sorted ascending
    std::vector<uint64_t> okey(B.n_search_items);
    for (size_t i = 0; i < okey.size(); ++i) okey[i] = ((uint64_t)(~items[i].cost) << 32) | (uint64_t)i;
    std::sort(okey.begin(), okey.end());
    // launch entries: a split pair twice (parts 0 and 1, adjacent)
    std::vector<uint32_t> order;
    order.reserve(2 * okey.size());
    for (size_t i = 0; i < okey.size(); ++i) {
        const uint32_t it = (uint32_t)(okey[i] & 0xFFFFFFFFu);
        order.push_back(it);
        if ((items[it].step >> 8) > 1) order.push_back(it | 0x80000000u);  // part 1
    }
    B.n_units = (uint32_t)order.size();
    // fusion stage: the largest target of the batch (new keyframes, and neighbours for
    // forward fusion)
    int fuse_n = 0;
    for (uint32_t i = B.n_search_items; i < items.size(); ++i) fuse_n = std::max(fuse_n, (int)items[i].nt);
    B.fsn = (uint32_t)std::max(16, (fuse_n + 15) & ~15);
    // the entry form's list (batches whose search has every form): room for four candidates a
    // query visit (at least 1 M), unless a test fixes it; the tuner grows it to a batch's count
    const bool entry_ok = sp.mode != TM_MODE_PER_PAIR && !(sp.epipole_px > 0.0f) && sp.dense_min <= 0;
    const uint32_t ent_cap = !entry_ok ? 0u
        : c->entry_cap > 0 ? (uint32_t)std::min<long long>(c->entry_cap, kEntryCapMax)
        : (uint32_t)std::min<size_t>(std::max<size_t>(B.ent_cap, std::max<size_t>(size_t(1) << 20, 4 * dq)), kEntryCapMax);
    // device buffers
    const size_t ni = std::max<size_t>(1, items.size());
    const size_t nm = std::max<int>(1, mps.n);
    const size_t nsi = std::max<size_t>(1, B.n_search_items), nun = std::max<size_t>(1, B.n_units);
    cudaError_t e;
    if ((e = B.items.reserve(align128(ni * sizeof(WorkItem)) + nun * sizeof(WorkItem))) ||
        (e = B.counts.reserve(ni * 4)) || (e = B.item_cmp.reserve(ni * 4)) ||
        (e = B.offsets.reserve((ni + 2) * 4)) ||
        (e = B.ncmp.reserve(24)) || (e = B.counters.reserve(16)) ||
        (e = B.padded.reserve(std::max<size_t>(1, pad) * sizeof(Out3))) ||
        (e = B.dense.reserve(std::max<size_t>(1, pad) * sizeof(Out3))) ||
        (e = B.masks.reserve(std::max<size_t>(16, mask_bytes))) ||
        (e = B.mp_pos.reserve(nm * 12)) || (e = B.mp_normal.reserve(nm * 12)) ||
        (e = B.mp_desc.reserve(nm * 32)) || (e = B.mp_min.reserve(nm * 4)) ||
        (e = B.mp_max.reserve(nm * 4)) || (e = B.mp_skip.reserve(nm)) ||
        (e = B.dres.reserve(std::max<size_t>(1, dq) * 8)) ||
        (e = B.work.reserve(16)) ||
        (e = B.acc.reserve(std::max<size_t>(1, dq) * 8)) ||
        (e = B.pconst.reserve(nsi * kPairConst * 4)) || (e = B.pwords.reserve(std::max<uint32_t>(64, tq) / 32 * 8)) ||
        (e = B.pepos.reserve(std::max<uint32_t>(64, tq) * 2)) ||
        (e = B.pwin.reserve(std::max<uint32_t>(64, tq) * 4)) || (e = B.pacc.reserve(nsi * 8)) ||
        (e = B.pdone.reserve(nsi * 4)) || (e = B.povf.reserve(nsi * 4)) ||
        (blk && (e = B.mp_block.reserve(std::max<uint64_t>(16, blk_bytes)))) ||
        (entry_ok && (e = B.ents.reserve(size_t(ent_cap) * 8))) ||
        (tri && ((e = B.points.reserve(std::max<size_t>(1, B.search_pad) * 12)) ||
                 (e = B.point_ok.reserve(std::max<size_t>(1, B.search_pad))))))
        return cuda_fail(e, "batch buffers");
    B.ent_cap = ent_cap;
    if (B.pointers() != before && (B.graph || B.graph_timed)) {
        if (B.graph) cudaGraphExecDestroy(B.graph);
        if (B.graph_timed) cudaGraphExecDestroy(B.graph_timed);
        B.graph = B.graph_timed = nullptr;
    }
    // one pinned staging area, one transfer for both tables: items (logical order), then the
    // search items again in launch order (each with its logical index)
    for (uint32_t k = 0; k < B.n_search_items; ++k) items[k].idx = k;
    const size_t o_order = align128(ni * sizeof(WorkItem));
    const size_t stage = o_order + order.size() * sizeof(WorkItem);
    if ((e = B.h_stage.reserve(std::max<size_t>(stage, 128)))) return cuda_fail(e, "pinned staging");
    unsigned char *h = static_cast<unsigned char *>(B.h_stage.p);
    if (!items.empty()) memcpy(h, items.data(), items.size() * sizeof(WorkItem));
    WorkItem *hs = reinterpret_cast<WorkItem *>(h + o_order);
    for (size_t k = 0; k < order.size(); ++k) {
        hs[k] = items[order[k] & 0x7FFFFFFFu];
        if (order[k] & 0x80000000u) hs[k].step |= 1u;  // part 1 of a split pair
    }
    if (!items.empty() &&
        (e = cudaMemcpyAsync(B.items.p, h, order.empty() ? items.size() * sizeof(WorkItem) : stage, cudaMemcpyHostToDevice, s)))
        return cuda_fail(e, "work list upload");
    if (mask_bytes && (e = cudaMemcpyAsync(B.masks.p, in->masks, mask_bytes, cudaMemcpyDefault, s)))
        return cuda_fail(e, "mask upload");
    // a one-shot batch forks its search branch here (it needs the work list, the masks and the
    // staged keyframes, not the map points) unless a neighbour enters with the batch
    if (B.early_fork) {
        if ((st = ensure_branches(B))) return st;
        if (!(B.n_new > 0 && B.nbr_new)) {
            if ((e = cudaEventRecord(B.pfork, s))) return cuda_fail(e, "search branch");
            B.forked = true;
        }
    }
    const cudaStream_t ms = s;
    if (mps.n > 0 && !mp_copied && (e = upload_mps(ms))) return cuda_fail(e, "map point upload");
    BatchArgs &A = B.args;
    A.items = static_cast<const WorkItem *>(B.items.p);
    A.n_items = B.n_items;
    A.n_search = B.n_search_items;
    A.n_bwd = B.n_bwd_items;
    A.sitems = reinterpret_cast<const WorkItem *>(static_cast<unsigned char *>(B.items.p) + align128(ni * sizeof(WorkItem)));
    A.counters = static_cast<uint32_t *>(B.counters.p);
    A.masks = static_cast<const uint8_t *>(B.masks.p);
    const unsigned char *db = static_cast<const unsigned char *>(B.mp_block.p);
    A.mp_pos = blk ? reinterpret_cast<const float *>(db + boff[0]) : static_cast<const float *>(B.mp_pos.p);
    A.mp_normal = blk ? reinterpret_cast<const float *>(db + boff[1]) : static_cast<const float *>(B.mp_normal.p);
    A.mp_min = blk ? reinterpret_cast<const float *>(db + boff[3]) : static_cast<const float *>(B.mp_min.p);
    A.mp_max = blk ? reinterpret_cast<const float *>(db + boff[4]) : static_cast<const float *>(B.mp_max.p);
    A.n_mp = (uint32_t)std::max(0, mps.n);
    A.mp_desc = blk ? reinterpret_cast<const uint4 *>(db + boff[2]) : static_cast<const uint4 *>(B.mp_desc.p);
    A.mp_skip = !(mps.n > 0 && mps.skip) ? nullptr
        : blk ? db + boff[5] : static_cast<const uint8_t *>(B.mp_skip.p);
    A.padded = static_cast<Out3 *>(B.padded.p);
    A.counts = static_cast<uint32_t *>(B.counts.p);
    A.offsets = static_cast<uint32_t *>(B.offsets.p);
    A.ncmp = static_cast<unsigned long long *>(B.ncmp.p);
    A.dense = static_cast<Out3 *>(B.dense.p);
    A.item_cmp = static_cast<uint32_t *>(B.item_cmp.p);
    A.fsn = B.fsn;
    A.sp = to_const(sp);
    A.fp.chi2 = fp.chi2;
    A.fp.hamming_max = fp.hamming_max;
    A.fp.radius_scale = fp.radius_scale;
    A.cam = c->camc;
    A.cap = c->cap;
    A.L = SlotLayout::make(c->cap);
    A.wait_limit = c->wait_limit;
    A.starve = c->starve;
    A.sn = B.smem_n;
    A.dres = static_cast<uint2 *>(B.dres.p);
    A.acc = static_cast<uint2 *>(B.acc.p);
    A.pconst = static_cast<float *>(B.pconst.p);
    A.pwords = static_cast<uint2 *>(B.pwords.p);
    A.pepos = static_cast<uint16_t *>(B.pepos.p);
    A.pwin = static_cast<uint32_t *>(B.pwin.p);
    A.pacc = static_cast<uint32_t *>(B.pacc.p);
    A.pdone = static_cast<uint32_t *>(B.pdone.p);
    A.n_units = B.n_units;
    A.work = static_cast<uint32_t *>(B.work.p);
    if ((e = cudaMemsetAsync(B.work.p, 0, 4, s))) return cuda_fail(e, "work counter");
    A.triangulate = tri ? 1 : 0;
    A.tri_cos_max = tri ? tri->cos_parallax_max : 0.0;
    A.tri_chi2 = tri ? tri->chi2 : 0.0;
    A.tri_ratio = tri ? tri->ratio_factor : 0.0;
    A.points = static_cast<float *>(B.points.p);
    A.point_ok = static_cast<uint8_t *>(B.point_ok.p);
    // dense kernel: at most one wave of three CTAs per SM over the pairs (a CTA takes every
    // dsplit-th dense run of its pair)
    B.dsplit_base = (uint32_t)std::max(1, std::min(64, 3 * c->num_sms / (int)nsi));
    A.dsplit = B.dsplit_base;
    B.user_dense_min = sp.dense_min;
    B.sp = sp;
    B.fp = fp;
    rollback.armed = false;
    return TM_OK;
}

std::vector<void *> BatchBuf::pointers() const {
    return {items.p, masks.p, mp_pos.p, mp_normal.p, mp_desc.p, mp_min.p, mp_max.p,
            mp_skip.p, padded.p, counts.p, item_cmp.p, offsets.p, ncmp.p, counters.p, dense.p, dres.p, acc.p, pconst.p,
            pwords.p, pepos.p, work.p, points.p,
            point_ok.p, pwin.p, pacc.p, pdone.p, ents.p, povf.p, mp_block.p};
}

// Takes the keyframes that entered the store with batch B out again (failed call).
static void drop_new_keyframes(tm_ctx *c, BatchBuf &B, const tm_batch_inputs *in) {
    if (!in || B.n_new <= 0) return;
    for (int k = 0; k < B.n_new; ++k) {
        auto it = c->ids.find(in->new_ids[k]);
        if (it == c->ids.end()) continue;
        c->free_slots.push_back(it->second);
        c->ids.erase(it);
    }
    B.n_new = 0;
}

// Records a stage-boundary event; inside a stream capture it must become an event-record
// node of the graph, which needs the external flag.
static cudaError_t record_stage(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e) return e;
    return cudaEventRecordWithFlags(ev, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                               : cudaEventRecordDefault);
}

// Enqueue the batch pipeline as a graph of kernels only (no memset or event nodes, which cost
// several microseconds each inside a graph).  Two branches:
//   search: search_kernel (one CTA per pair) on `paux`, at high priority; it reads new keyframes
//           from their staged arrays, so it runs beside their ingest (unless a neighbour enters
//           with the batch: then it starts after the ingest);
//   store:  ingest of new keyframes -> fusion (needs their grids), on s, at low priority;
// each branch then compacts its own records (offsets, dense output, comparison totals, status:
// the search part from record 0, then the triangulation of its matches; the fusion part from
// record search_pad), and the store branch awaits the search branch.  `threads` = threads per
// search CTA.  With `timed`, events E0..E5 mark: start, search done, ingest done, fusion done,
// both copies done, search start (on the search branch, right before the kernel); E6 (with
// dense node blocks) between the dense and the search kernel.
tm_status tmap::enqueue_fused(tm_ctx *c, BatchBuf &B, int threads, int lanes, cudaStream_t s, bool timed) {
    cudaError_t e;
    B.threads = threads;
    B.lanes = lanes;
    // the launch choices in effect: the tuner's (B.knobs) unless a test hook fixes one
    BatchArgs &KA = B.args;
    KA.qpl = (uint32_t)(c->force_qpl ? c->force_qpl : B.knobs.qpl);
    KA.persist = (uint32_t)(c->force_persist >= 0 ? c->force_persist : B.knobs.persist);
    KA.l2_prefetch = (uint32_t)(c->force_prefetch >= 0 ? c->force_prefetch : B.knobs.prefetch);
    if (B.user_dense_min < 0) KA.sp.dense_min = B.knobs.dense_min;
    KA.dsplit = std::max(1u, B.dsplit_base / (uint32_t)std::max(1, B.knobs.dsplit_div));
    if (KA.qpl == 4 && !B.ent_cap) KA.qpl = 2;  // (the batch has no entry list)
    KA.ents = static_cast<uint2 *>(B.ents.p);
    KA.nents = static_cast<uint32_t *>(B.work.p) + 1;
    KA.ent_cap = B.ent_cap;
    KA.povf = static_cast<uint32_t *>(B.povf.p);
    search_form(KA);
    const int per_sm = search_ctas_per_sm(KA);
    if (per_sm < 1) return fail(TM_ERR_INVALID_ARG, "search kernel does not fit");
    B.ctas = KA.persist ? std::min((int)B.n_units, per_sm * c->num_sms) : (int)B.n_units;
    if (timed && !B.ev[0])
        for (cudaEvent_t &ev : B.ev)
            if ((e = cudaEventCreate(&ev))) return cuda_fail(e, "events");
    tm_status bst = ensure_branches(B);
    if (bst) return bst;
    auto mark = [&](int k, cudaStream_t st) { return timed ? record_stage(B.ev[k], st) : cudaSuccess; };
    // the search branch is the critical path: its CTAs are placed before the store branch's
    // when SMs free up (priorities within the device's range; `hi` is numerically lowest)
    int lo_p = 0, hi_p = 0;
    if ((e = cudaDeviceGetStreamPriorityRange(&lo_p, &hi_p))) return cuda_fail(e, "priorities");
    // which branch's CTAs the scheduler places first when SMs free up: the store branch
    // (ingest -> fusion) or the search branch
    int sp_ = hi_p, st_ = lo_p;
    const int bprio = c->branch_prio >= 0 ? c->branch_prio : B.knobs.bprio;
    if (bprio == 1) std::swap(sp_, st_);
    if (bprio == 2) sp_ = st_ = 0;
    if ((e = mark(0, s))) return cuda_fail(e, "event");
    const bool after_ingest = B.n_new > 0 && B.nbr_new;
    const bool forked = B.forked, mp_async = B.mp_async;  // set by prepare_batch, for this enqueue only
    B.forked = B.mp_async = false;
    if (!after_ingest && !forked && (e = cudaEventRecord(B.pfork, s))) return cuda_fail(e, "search branch");
    if (B.n_new > 0 && (e = launch_ingest(B.ingest_args, s, st_))) return cuda_fail(e, "ingest kernel");
    if (B.ingest_done && (e = cudaEventRecord(B.ingest_done, s))) return cuda_fail(e, "event");
    if ((e = mark(2, s))) return cuda_fail(e, "event");
    if (after_ingest && (e = cudaEventRecord(B.pfork, s))) return cuda_fail(e, "search branch");
    if ((e = cudaStreamWaitEvent(B.paux, B.pfork, 0)) || (e = mark(5, B.paux)) ||
        (e = launch_prep(B.args, B.paux, sp_)) || (e = mark(7, B.paux)) ||
        (e = launch_dense(B.args, B.paux, sp_)) ||
        (B.args.sp.dense_min > 0 && B.n_search_items > 0 && (e = mark(6, B.paux))) ||
        (e = launch_search(B.args, B.ctas, B.paux, sp_)) || (e = mark(1, B.paux)))
        return cuda_fail(e, "search kernel");
    // each branch compacts its own records (about one warp per item, 32 per CTA, at most one
    // CTA per SM): the search part on the search branch (then the triangulation of its
    // matches), the fusion part on the store branch, from record search_pad on
    const uint32_t nfi = B.n_items - B.n_search_items;
    auto copy_ctas = [&](uint32_t n) { return (int)std::max<uint32_t>(1, std::min<uint32_t>((n + 31) / 32, c->num_sms)); };
    if ((e = launch_copy(B.args, 0, 0u, copy_ctas(B.n_search_items), B.paux)) || (e = launch_tri(B.args, B.paux)) ||
        (e = cudaEventRecord(B.join, B.paux)))
        return cuda_fail(e, "search copy");
    if (mp_async && (e = cudaStreamWaitEvent(s, B.mready, 0))) return cuda_fail(e, "map points");
    if ((nfi && (e = launch_fuse(B.args, s, st_))) || (e = mark(3, s)) ||
        (e = launch_copy(B.args, 1, (uint32_t)B.search_pad, copy_ctas(nfi), s)) ||
        (e = cudaStreamWaitEvent(s, B.join, 0)))
        return cuda_fail(e, "fusion kernel");
    if ((e = mark(4, s))) return cuda_fail(e, "event");
    return TM_OK;
}

// Enqueue the plain per-pair form of the same batch.
tm_status tmap::enqueue_plain(tm_ctx *c, BatchBuf &B, int lanes, cudaStream_t s) {
    cudaError_t e;
    const size_t scr_bytes = pair_scratch_bytes(c->cap);
    const int max_mp = (int)B.total_pad;  // a step's map points never exceed the padded total
    if ((e = B.scratch.reserve(scr_bytes + align128(size_t(std::max(1, max_mp)) * 4))))
        return cuda_fail(e, "plain scratch");
    PairScratch scr = pair_scratch_at(B.scratch.p, c->cap);
    if (B.n_new > 0 && (e = launch_ingest(B.ingest_args, s))) return cuda_fail(e, "ingest kernel");
    if (B.ingest_done && (e = cudaEventRecord(B.ingest_done, s))) return cuda_fail(e, "event");
    uint32_t *res = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(B.scratch.p) + scr_bytes);
    if ((e = cudaMemsetAsync(scr.running, 0, 8, s)) || (e = cudaMemsetAsync(B.ncmp.p, 0, 24, s)))
        return cuda_fail(e, "reset");
    B.lanes = lanes;
    const std::vector<WorkItem> &items = B.h_items;
    uint32_t *offs = static_cast<uint32_t *>(B.offsets.p);
    unsigned long long *ncmp = static_cast<unsigned long long *>(B.ncmp.p);
    const SearchConst sp = to_const(B.sp);
    for (uint32_t i = 0; i < B.n_search_items; ++i) {
        const WorkItem &w = items[i];
        const int qn = B.item_nq[i], tn = B.item_nt[i];
        const uint8_t *mq = w.a == kNone ? nullptr : B.args.masks + w.a;
        const uint8_t *mt = w.b == kNone ? nullptr : B.args.masks + w.b;
        if ((e = launch_pair_plain(w.q, w.t, mq, mt, qn, tn, c->cap, sp, c->camc, scr, B.args.dense,
                                   offs + i, ncmp, lanes, s, w.mdepth)))
            return cuda_fail(e, "plain pair");
    }
    // the search part's total; the fusion part's records from record search_pad on, its offsets
    // relative to that (the layout of the fused form's two copies)
    if ((e = cudaMemcpyAsync(offs + B.n_items, scr.running, 4, cudaMemcpyDeviceToDevice, s)) ||
        (e = cudaMemsetAsync(scr.running, 0, 4, s)))
        return cuda_fail(e, "plain search total");
    Out3 *fdense = B.args.dense + B.search_pad;
    for (int k = 0; k < B.n_steps; ++k) {
        const int f0 = B.step_fuse_item[k], f1 = B.step_fuse_item[k + 1];
        if (f0 == f1) continue;
        const WorkItem &w = items[f0];
        const uint32_t begin = w.a;
        uint32_t n = 0;
        for (int f = f0; f < f1; ++f) n += items[f].b;
        if ((e = launch_fuse_plain(w.q, c->cap, B.args.mp_pos + 3 * (size_t)begin,
                                   B.args.mp_normal + 3 * (size_t)begin, B.args.mp_desc + 2 * (size_t)begin,
                                   B.args.mp_min + begin, B.args.mp_max + begin,
                                   B.args.mp_skip ? B.args.mp_skip + begin : nullptr, (int)n, B.args.fp,
                                   c->camc, res, fdense, scr.running, offs + f0, ncmp + 1, s)))
            return cuda_fail(e, "plain fuse");
    }
    for (int p = 0; p < B.n_pairs && B.any_fwd; ++p) {  // forward fusion, pair by pair
        const int f0 = B.pair_fwd_item[p], f1 = B.pair_fwd_item[p + 1];
        if (f0 == f1) continue;
        const WorkItem &w = items[f0];
        const uint32_t begin = w.a;
        uint32_t n = 0;
        for (int f = f0; f < f1; ++f) n += items[f].b;
        if ((e = launch_fuse_plain(w.q, c->cap, B.args.mp_pos + 3 * (size_t)begin,
                                   B.args.mp_normal + 3 * (size_t)begin, B.args.mp_desc + 2 * (size_t)begin,
                                   B.args.mp_min + begin, B.args.mp_max + begin,
                                   w.skip != kNone ? B.args.masks + w.skip : nullptr, (int)n, B.args.fp,
                                   c->camc, res, fdense, scr.running, offs + f0, ncmp + 2, s)))
            return cuda_fail(e, "plain forward fuse");
    }
    if ((e = cudaMemcpyAsync(offs + B.n_items + 1, scr.running, 4, cudaMemcpyDeviceToDevice, s)))
        return cuda_fail(e, "plain total");
    if ((e = launch_tri(B.args, s))) return cuda_fail(e, "triangulation kernel");
    return TM_OK;
}

// Download results of the last run of B into r (host offsets; matches host or device).
tm_status tmap::fetch_results(tm_ctx *c, BatchBuf &B, tm_batch_result *r, cudaStream_t s, double *t_counts) {
    cudaError_t e;
    // item offsets, then the search part's total and the fusion part's (each part's offsets
    // relative to its base: record 0, record search_pad)
    const size_t nio = (size_t)B.n_items + 2;
    if ((e = B.h_out.reserve((nio + 2) * 4 + 48))) return cuda_fail(e, "pinned results");
    uint32_t *ho = static_cast<uint32_t *>(B.h_out.p);
    unsigned long long *hc = reinterpret_cast<unsigned long long *>(ho + ((nio + 1) & ~size_t(1)));
    uint32_t *hs = reinterpret_cast<uint32_t *>(hc + 3);
    if ((e = cudaMemcpyAsync(ho, B.offsets.p, nio * 4, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(hc, B.ncmp.p, 24, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(hs, static_cast<uint32_t *>(B.counters.p) + 2, 8, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "results");
    *(t_counts ? t_counts : &c->t_counts) = tm_now();
    // (a part with no items launched no copy: its words are not this run's)
    const bool has_s = B.n_search_items > 0, has_f = B.n_items > B.n_search_items;
    const uint32_t status = (has_s ? hs[0] : 0u) | (has_f ? hs[1] : 0u);
    if (B.sp.mode != TM_MODE_PER_PAIR && (status & kStatusTimeout))
        return fail(TM_ERR_TIMEOUT, "a bulk copy into shared memory or a tensor-core product did not complete in time");
    const uint32_t search_total = has_s ? ho[B.n_items] : 0u, fuse_total = has_f ? ho[B.n_items + 1] : 0u;
    // offset of a fusion item in the fusion part (its end for n_items)
    auto foff = [&](int k) -> uint32_t { return k < (int)B.n_items ? ho[k] : fuse_total; };
    const uint32_t bwd_end = foff((int)(B.n_search_items + B.n_bwd_items));
    const size_t nf = bwd_end, nw = fuse_total - bwd_end;
    r->n_matches = search_total;
    r->n_fuse = nf;
    r->n_fwd = nw;
    r->n_comparisons_search = has_s ? hc[0] : 0ull;
    r->n_comparisons_fuse = has_f ? hc[1] : 0ull;
    r->n_comparisons_fwd = has_f ? hc[2] : 0ull;
    if (B.args.triangulate && (!r->points || !r->point_ok))
        return fail(TM_ERR_INVALID_ARG, "triangulation needs points and point_ok result buffers");
    if (search_total > r->match_cap || nf > r->fuse_cap || (nw && (!r->fwd || nw > r->fwd_cap)))
        return fail(TM_ERR_CAPACITY, "result buffers too small: %u matches (cap %zu), %zu fusion candidates (cap %zu), "
                    "%zu forward-fusion candidates (cap %zu)", search_total, r->match_cap, nf, r->fuse_cap, nw,
                    r->fwd ? r->fwd_cap : (size_t)0);
    if (r->pair_offsets) {
        for (int p = 0; p < B.n_pairs; ++p) r->pair_offsets[p] = (int32_t)ho[p];
        r->pair_offsets[B.n_pairs] = (int32_t)search_total;
    }
    if (r->fuse_offsets)
        for (int k = 0; k <= B.n_steps; ++k) r->fuse_offsets[k] = (int32_t)foff(B.step_fuse_item[k]);
    if (r->fuse_offsets && B.n_steps > 0) {
        // steps without map points start where the next step starts
        for (int k = B.n_steps - 1; k >= 0; --k)
            if (B.step_fuse_item[k] == B.step_fuse_item[k + 1]) r->fuse_offsets[k] = r->fuse_offsets[k + 1];
    }
    if (r->fwd_offsets) {
        for (int p = 0; p <= B.n_pairs; ++p) r->fwd_offsets[p] = (int32_t)(foff(B.pair_fwd_item[p]) - bwd_end);
        // pairs without forward items start where the next pair starts
        for (int p = B.n_pairs - 1; p >= 0; --p)
            if (B.pair_fwd_item[p] == B.pair_fwd_item[p + 1]) r->fwd_offsets[p] = r->fwd_offsets[p + 1];
    }
    const Out3 *d = static_cast<const Out3 *>(B.dense.p), *df = d + B.search_pad;
    if (search_total && (e = cudaMemcpyAsync(r->matches, d, search_total * sizeof(Out3), cudaMemcpyDefault, s)))
        return cuda_fail(e, "matches download");
    if (nf && (e = cudaMemcpyAsync(r->fuse, df, nf * sizeof(Out3), cudaMemcpyDefault, s)))
        return cuda_fail(e, "fusion download");
    if (nw && (e = cudaMemcpyAsync(r->fwd, df + bwd_end, nw * sizeof(Out3), cudaMemcpyDefault, s)))
        return cuda_fail(e, "forward fusion download");
    if (B.args.triangulate && search_total &&
        ((e = cudaMemcpyAsync(r->points, B.points.p, (size_t)search_total * 12, cudaMemcpyDefault, s)) ||
         (e = cudaMemcpyAsync(r->point_ok, B.point_ok.p, search_total, cudaMemcpyDefault, s))))
        return cuda_fail(e, "points download");
    if ((e = cudaStreamSynchronize(s))) return cuda_fail(e, "results");
    return TM_OK;
}

// ------------------------------------------------------------------------- tuning


// Launch shape of the search kernel: 256 threads per CTA (five per SM).
int tmap::default_threads(const tm_ctx *, const BatchBuf &) { return 256; }

// Layout of the regime keys in a tuning cache file (its first line).
static constexpr int kTuneVersion = 2;

void tmap::load_tuning(tm_ctx *c, const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return;
    int key, version = 0;
    Knobs k;
    // (a file of another key layout is ignored: its choices would be taken for other regimes)
    if (fscanf(f, "tm-tune %d", &version) != 1 || version != kTuneVersion) {
        fclose(f);
        return;
    }
    while (fscanf(f, "%d %d %d %d %d %d %d", &key, &k.qpl, &k.persist, &k.prefetch, &k.bprio, &k.dense_min,
                  &k.dsplit_div) == 7)
        if (k.qpl >= 1 && k.qpl <= 4 && k.dsplit_div >= 1) c->tuned_knobs[key] = k;
    fclose(f);
}

static void save_tuning(tm_ctx *c) {
    const char *path = getenv("TM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "tm-tune %d\n", kTuneVersion);
    for (auto &kv : c->tuned_knobs) {
        const Knobs &k = kv.second;
        fprintf(f, "%d %d %d %d %d %d %d\n", kv.first, k.qpl, k.persist, k.prefetch, k.bprio, k.dense_min, k.dsplit_div);
    }
    fclose(f);
}

// Density class of a batch: log2 of the mean candidates per query keypoint.
static int density_key(uint64_t ncmp, uint64_t queries) {
    if (!queries) return 0;
    double r = (double)ncmp / (double)queries;
    return (int)std::lround(std::log2(std::max(r, 0.25)) * 2.0);
}

static uint64_t batch_queries(tm_ctx *c, const BatchBuf &B, const tm_step *steps) {
    uint64_t q = 0;
    for (int k = 0; k < B.n_steps; ++k)
        q += (uint64_t)c->slots[c->ids[steps[k].kf_id]].n * (uint64_t)steps[k].n_nbrs;
    return q;
}

// Picks the launch choices of a prepared batch (B.knobs): cached by batch regime, else measured
// by coordinate descent (each choice in turn, the others held at the best so far; a choice is
// timed over three enqueues after a warm-up).  The regime: density class (comparisons per query
// of a first run), pairs fewer than SMs, dense blocks left to the tuner.  Results never depend
// on the choices.
tm_status tmap::tune_batch(tm_ctx *c, BatchBuf &B, const tm_step *steps, cudaStream_t s, bool measure) {
    tm_status st;
    B.threads = 256;
    B.lanes = c->def_lanes;
    B.knobs = Knobs{};
    B.tuned = false;
    if ((st = enqueue_fused(c, B, 256, c->def_lanes, s))) return st;
    unsigned long long hc[2];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hc, B.ncmp.p, 16, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "tuning");
    const bool dense_auto = B.user_dense_min < 0 && B.n_search_items > 0;
    // dense blocks off, on at the caller's dense_min, or left to the tuner; epipole rejection:
    // with dense blocks on or epipole rejection the search has one group form only, so such
    // batches neither tune the form nor share choices with batches that have all of them
    const int dense_mode = dense_auto ? 2 : (B.user_dense_min > 0 ? 1 : 0);
    const bool epi_rej = B.sp.epipole_px > 0.0f;
    const bool forms = dense_mode != 1 && !epi_rej;
    const int key = (((density_key(hc[0], batch_queries(c, B, steps)) * 2 +
                       ((int)B.n_search_items < c->num_sms ? 1 : 0)) * 3 + dense_mode) * 2) + (epi_rej ? 1 : 0);
    // the entry form's list: room for this batch's entries (its comparisons), so that a plan
    // that takes the form never falls back to rounds
    if (forms && B.ent_cap && !c->entry_cap && hc[0] > B.ent_cap) {
        const size_t want = std::min<size_t>(size_t(hc[0] + hc[0] / 16), size_t(kEntryCapMax));
        if ((e = B.ents.reserve(want * 8))) return cuda_fail(e, "entry list");
        B.ent_cap = (uint32_t)want;
    }
    auto it = c->tuned_knobs.find(key);
    if (it != c->tuned_knobs.end()) {
        B.knobs = it->second;
        B.tuned = true;
        return TM_OK;
    }
    if (!measure) return TM_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a choice is timed as the plan will run it: captured into a graph, replayed once to warm
    // up, then the median of up to 16 replays (at least ~1 ms of them, so that a small batch's
    // choices are told apart), each between events on the stream and each after 256 MB
    // written (L2 flushed: a batch's inputs are not in L2 when it runs)
    void *flush = nullptr;
    const size_t flush_bytes = size_t(256) << 20;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;  // (timed with a warm L2 then)
    }
    auto time_of = [&](const Knobs &k, float &ms) -> tm_status {
        B.knobs = k;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (ce) return cuda_fail(ce, "tuning capture");
        tm_status r = enqueue_fused(c, B, 256, c->def_lanes, c->capture_stream);
        ce = cudaStreamEndCapture(c->capture_stream, &g);
        if (!r && ce) r = cuda_fail(ce, "tuning capture");
        if (!r && (ce = cudaGraphInstantiate(&x, g, 0))) r = cuda_fail(ce, "tuning graph");
        if (g) cudaGraphDestroy(g);
        if (r) return r;
        ms = 0.0f;
        float t = 0.0f;
        std::vector<float> ts;
        for (int rep = 0, reps = 2; rep < reps; ++rep) {
            if ((flush && (ce = cudaMemsetAsync(flush, rep & 0xFF, flush_bytes, s))) ||
                (ce = cudaEventRecord(e0, s)) || (ce = cudaGraphLaunch(x, s)) || (ce = cudaEventRecord(e1, s)) ||
                (ce = cudaEventSynchronize(e1)) || (ce = cudaEventElapsedTime(&t, e0, e1))) {
                r = cuda_fail(ce, "tuning replay");
                break;
            }
            if (rep == 0) {  // the warm-up sets how many replays follow
                reps = 1 + std::max(3, std::min(16, (int)std::ceil(1.0f / std::max(t, 1e-3f))));
                continue;
            }
            ts.push_back(t);
        }
        if (!ts.empty()) {
            std::nth_element(ts.begin(), ts.begin() + ts.size() / 2, ts.end());
            ms = ts[ts.size() / 2];
        }
        cudaGraphExecDestroy(x);
        return r;
    };
    Knobs best{};
    float tbest = 0.0f;
    st = time_of(best, tbest);
    const bool both_branches = B.n_search_items > 0 && (B.n_new > 0 || B.n_items > B.n_search_items);
    for (int knob = 0; knob < 6 && !st; ++knob) {
        std::vector<Knobs> alts;
        Knobs k = best;
        switch (knob) {
            case 0:
                if (!c->force_qpl && forms)
                    for (int qf : {2, 1, 3, 4})
                        if (qf != best.qpl) { k.qpl = qf; alts.push_back(k); }
                break;
            case 1: if (c->force_persist < 0 && forms) { k.persist = !best.persist; alts.push_back(k); } break;
            case 2: if (c->force_prefetch < 0) { k.prefetch = !best.prefetch; alts.push_back(k); } break;
            case 3:
                if (c->branch_prio < 0 && both_branches)
                    for (int bp : {0, 1, 2})  // search first, store first, equal
                        if (bp != best.bprio) { k.bprio = bp; alts.push_back(k); }
                break;
            case 4:
                if (dense_auto)
                    for (int dm : {64, 32, 128})
                        if (dm != best.dense_min) { k.dense_min = dm; alts.push_back(k); }
                break;
            case 5: if (best.dense_min > 0 && B.dsplit_base > 1) { k.dsplit_div = 2; alts.push_back(k); } break;
        }
        for (const Knobs &a : alts) {
            float t = 0.0f;
            if ((st = time_of(a, t))) break;
            if (t < tbest) {
                tbest = t;
                best = a;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
    if (st) return st;
    B.knobs = best;
    B.tuned = true;
    c->tuned_knobs[key] = best;
    save_tuning(c);
    return TM_OK;
}

// ------------------------------------------------------------------------- one-shot calls

static tm_status run_batch_locked(tm_ctx *c, const tm_step *steps, int n_steps,
                                  const tm_batch_inputs *in, const tm_search_params &sp,
                                  const tm_fuse_params &fp, tm_batch_result *res, cudaStream_t s) {
    Range range("tm_batch_run");
    BatchBuf &B = c->batch;
    B.early_fork = sp.mode != TM_MODE_PER_PAIR;  // one-shot: nothing of this enqueue is captured
    tm_status st;
    const double t0 = tm_now();
    c->t_counts = 0;
    {
        Range r("prepare_batch (work list, uploads)");
        st = prepare_batch(c, B, steps, n_steps, in, sp, fp, s);
    }
    B.early_fork = false;
    const double t1 = tm_now();
    if (st) {
        // copies of the caller's arrays may be in flight: done before the call returns
        if (B.mcopy) cudaStreamSynchronize(B.mcopy);
        cudaStreamSynchronize(s);
        return st;
    }
    if (sp.mode == TM_MODE_PER_PAIR) {
        st = enqueue_plain(c, B, sp.lanes_per_query ? sp.lanes_per_query : 1, s);
    } else {
        int th = default_threads(c, B), ln = c->def_lanes;
        if (sp.lanes_per_query) ln = sp.lanes_per_query;
        // the last tuned plan's launch choices (one-shot batches are not measured)
        B.knobs = c->last_staged == 1 ? c->last_knobs : Knobs{};
        st = enqueue_fused(c, B, th, ln, s);
    }
    const double t2 = tm_now();
    if (!st) {
        Range r("fetch_results (downloads, wait)");
        st = fetch_results(c, B, res, s);
    }
    const double t3 = tm_now(), tc = c->t_counts > 0 ? c->t_counts : t3;
    c->host_us[0] = 1e6 * (t1 - t0);
    c->host_us[1] = 1e6 * (t2 - t1);
    c->host_us[2] = 1e6 * (tc - t2);
    c->host_us[3] = 1e6 * (t3 - tc);
    if (st) {
        if (B.mcopy) cudaStreamSynchronize(B.mcopy);
        cudaStreamSynchronize(s);
        drop_new_keyframes(c, B, in);
    }
    return st;
}

extern "C" tm_status tm_batch_begin(tm_ctx *c, const tm_step *steps, int32_t n_steps,
                                    const tm_batch_inputs *in, const tm_search_params *sp,
                                    const tm_fuse_params *fp, uint64_t *ticket) {
    if (!c || !ticket) return fail(TM_ERR_INVALID_ARG, "tm_batch_begin: null argument");
    tm_search_params spd;
    tm_fuse_params fpd;
    tm_search_params_default(&spd);
    tm_fuse_params_default(&fpd);
    if (sp) spd = *sp;
    if (fp) fpd = *fp;
    Range range("tm_batch_begin");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    int k = -1;
    for (int q = 0; q < TM_BATCH_INFLIGHT; ++q)
        if (!c->async[q].ticket) { k = q; break; }
    if (k < 0) return fail(TM_ERR_BUSY, "tm_batch_begin: %d batches already in flight", TM_BATCH_INFLIGHT);
    tm_ctx::AsyncBatch &a = c->async[k];
    cudaError_t e;
    if (!a.s && ((e = cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking)) ||
                 (e = cudaEventCreateWithFlags(&a.ingested, cudaEventDisableTiming))))
        return cuda_fail(e, "async batch stream");
    BatchBuf &B = a.B;
    // this batch's uploads (its own buffers) start at once; its kernels wait for the ingest of
    // the batch begun before it (whose keyframes may be neighbours here)
    B.early_fork = spd.mode != TM_MODE_PER_PAIR;
    B.allow_pending = true;
    tm_status st = prepare_batch(c, B, steps, n_steps, in, spd, fpd, a.s);
    B.early_fork = false;
    B.allow_pending = false;
    const bool prepared = !st;  // (its new keyframes are then stored: taken out on failure)
    if (!st && c->async_last >= 0 && c->async[c->async_last].ticket) {
        // both branches: the stream's (ingest, fusion, copy) and the search branch, which a
        // one-shot batch forks early
        const cudaEvent_t prev = c->async[c->async_last].ingested;
        if ((e = cudaStreamWaitEvent(a.s, prev, 0)) || (B.paux && (e = cudaStreamWaitEvent(B.paux, prev, 0))))
            st = cuda_fail(e, "async batch order");
    }
    if (!st) {
        B.ingest_done = a.ingested;
        if (spd.mode == TM_MODE_PER_PAIR) {
            st = enqueue_plain(c, B, spd.lanes_per_query ? spd.lanes_per_query : 1, a.s);
        } else {
            int ln = c->def_lanes;
            if (spd.lanes_per_query) ln = spd.lanes_per_query;
            B.knobs = c->last_staged == 1 ? c->last_knobs : Knobs{};
            st = enqueue_fused(c, B, default_threads(c, B), ln, a.s);
        }
        B.ingest_done = nullptr;
    }
    if (st) {
        if (B.mcopy) cudaStreamSynchronize(B.mcopy);
        cudaStreamSynchronize(a.s);
        if (B.paux) cudaStreamSynchronize(B.paux);
        if (prepared) drop_new_keyframes(c, B, in);
        return st;
    }
    for (int sl : B.slots) c->slots[sl].refs++;
    a.new_ids.assign(in && in->n_new > 0 ? in->new_ids : nullptr, in && in->n_new > 0 ? in->new_ids + in->n_new : nullptr);
    a.ticket = c->async_next++;
    for (uint64_t id : a.new_ids) {
        auto it = c->ids.find(id);
        if (it != c->ids.end()) c->slots[it->second].pending = a.ticket;
    }
    c->async_last = k;
    *ticket = a.ticket;
    return TM_OK;
}

extern "C" tm_status tm_batch_finish(tm_ctx *c, uint64_t ticket, tm_batch_result *res) {
    if (!c || !res) return fail(TM_ERR_INVALID_ARG, "tm_batch_finish: null argument");
    Range range("tm_batch_finish");
    int k = -1;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (int q = 0; q < TM_BATCH_INFLIGHT; ++q)
            if (ticket && c->async[q].ticket == ticket && !c->async[q].finishing) { k = q; break; }
        if (k < 0) return fail(TM_ERR_NOT_FOUND, "tm_batch_finish: unknown ticket %llu", (unsigned long long)ticket);
        c->async[k].finishing = true;
    }
    cudaSetDevice(c->device);
    tm_ctx::AsyncBatch &a = c->async[k];
    BatchBuf &B = a.B;
    // the wait and the downloads use only the batch's own buffers and streams (its slot stays
    // taken until the end of this call), so they run without the context's lock: other threads
    // may begin batches, or finish other ones, meanwhile
    const double t0 = tm_now();
    double tcnt = 0;
    tm_status st = fetch_results(c, B, res, a.s, &tcnt);
    const double t1 = tm_now(), tc = tcnt > 0 ? tcnt : t1;
    if (st) {
        if (B.mcopy) cudaStreamSynchronize(B.mcopy);
        cudaStreamSynchronize(a.s);
    }
    std::lock_guard<std::mutex> lk(c->mu);
    c->host_us[0] = c->host_us[1] = 0.0;
    c->host_us[2] = 1e6 * (tc - t0);
    c->host_us[3] = 1e6 * (t1 - tc);
    for (int sl : B.slots) c->slots[sl].refs--;
    for (uint64_t id : a.new_ids) {
        auto it = c->ids.find(id);
        if (it != c->ids.end() && c->slots[it->second].pending == ticket) c->slots[it->second].pending = 0;
    }
    if (st && B.n_new > 0) {
        for (uint64_t id : a.new_ids) {
            auto it = c->ids.find(id);
            // (a keyframe that a batch begun later reads stays stored: its slot is in use)
            if (it == c->ids.end() || c->slots[it->second].refs > 0) continue;
            c->free_slots.push_back(it->second);
            c->ids.erase(it);
        }
    }
    B.n_new = 0;
    a.new_ids.clear();
    a.ticket = 0;
    a.finishing = false;
    return st;
}

extern "C" tm_status tm_batch_last_host_times(tm_ctx *c, double us[4]) {
    if (!c || !us) return fail(TM_ERR_INVALID_ARG, "tm_batch_last_host_times: null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    for (int k = 0; k < 4; ++k) us[k] = c->host_us[k];
    return TM_OK;
}

extern "C" tm_status tm_batch_run(tm_ctx *c, const tm_step *steps, int32_t n_steps,
                                  const tm_batch_inputs *in, const tm_search_params *sp,
                                  const tm_fuse_params *fp, tm_batch_result *res, void *stream) {
    if (!c || !res) return fail(TM_ERR_INVALID_ARG, "tm_batch_run: null argument");
    tm_search_params spd;
    tm_fuse_params fpd;
    tm_search_params_default(&spd);
    tm_fuse_params_default(&fpd);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return run_batch_locked(c, steps, n_steps, in, sp ? *sp : spd, fp ? *fp : fpd, res,
                            pick_stream(c, stream));
}

extern "C" tm_status tm_search_triangulation(tm_ctx *c, uint64_t kf, const uint64_t *nbrs,
                                             int32_t n_nbrs, const tm_search_params *params,
                                             const uint8_t *q_free, const uint8_t *nbr_free,
                                             tm_match *out, size_t cap, size_t *n_out,
                                             int32_t *pair_offsets, uint64_t *n_comparisons,
                                             void *stream) {
    if (!c || !n_out || (n_nbrs > 0 && (!nbrs || !pair_offsets)) || n_nbrs < 0)
        return fail(TM_ERR_INVALID_ARG, "tm_search_triangulation: bad arguments");
    tm_search_params sp;
    tm_fuse_params fp;
    tm_search_params_default(&sp);
    tm_fuse_params_default(&fp);
    if (params) sp = *params;
    Range range("tm_search_triangulation");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    auto it = c->ids.find(kf);
    if (it == c->ids.end()) return fail(TM_ERR_NOT_FOUND, "keyframe %llu not stored", (unsigned long long)kf);
    const int nq = c->slots[it->second].n;
    size_t nt_sum = 0;
    for (int k = 0; k < n_nbrs; ++k) {
        auto jt = c->ids.find(nbrs[k]);
        if (jt == c->ids.end()) return fail(TM_ERR_NOT_FOUND, "keyframe %llu not stored", (unsigned long long)nbrs[k]);
        nt_sum += (size_t)c->slots[jt->second].n;
    }
    // masks: [q_free | nbr_free], uploaded in one call when both come from one place
    std::vector<uint8_t> hm;
    tm_batch_inputs in{};
    tm_step st{};
    st.kf_id = kf;
    st.nbr_ids = nbrs;
    st.n_nbrs = n_nbrs;
    st.q_free_off = -1;
    st.nbr_free_off = -1;
    const bool dq = is_device_ptr(q_free), dn = is_device_ptr(nbr_free);
    if ((q_free && dq) || (nbr_free && dn)) {
        // device masks: gather them into the context's device scratch
        cudaError_t e = c->mask_scratch.reserve(nq + nt_sum + 16);
        if (e) return cuda_fail(e, "mask scratch");
        unsigned char *d = static_cast<unsigned char *>(c->mask_scratch.p);
        cudaStream_t s = pick_stream(c, stream);
        if (q_free && (e = cudaMemcpyAsync(d, q_free, nq, cudaMemcpyDefault, s))) return cuda_fail(e, "mask");
        if (nbr_free && (e = cudaMemcpyAsync(d + nq, nbr_free, nt_sum, cudaMemcpyDefault, s))) return cuda_fail(e, "mask");
        in.masks = d;
    } else {
        hm.resize(nq + nt_sum);
        if (q_free && nq) memcpy(hm.data(), q_free, nq);
        if (nbr_free && nt_sum) memcpy(hm.data() + nq, nbr_free, nt_sum);
        in.masks = hm.data();
    }
    in.mask_bytes = nq + nt_sum;
    if (q_free) st.q_free_off = 0;
    if (nbr_free) st.nbr_free_off = nq;
    std::vector<int32_t> fo(2);
    tm_batch_result r{};
    r.matches = out;
    r.match_cap = cap;
    r.pair_offsets = pair_offsets;
    r.fuse = nullptr;
    r.fuse_cap = 0;
    r.fuse_offsets = fo.data();
    tm_status s2 = run_batch_locked(c, &st, 1, &in, sp, fp, &r, pick_stream(c, stream));
    *n_out = r.n_matches;
    if (n_comparisons) *n_comparisons = r.n_comparisons_search;
    return s2;
}

extern "C" tm_status tm_fuse(tm_ctx *c, uint64_t kf, const tm_mappoint_view *mps,
                             const tm_fuse_params *params, tm_fuse_match *out, size_t cap,
                             size_t *n_out, uint64_t *n_comparisons, void *stream) {
    if (!c || !mps || !n_out) return fail(TM_ERR_INVALID_ARG, "tm_fuse: null argument");
    tm_search_params sp;
    tm_fuse_params fp;
    tm_search_params_default(&sp);
    tm_fuse_params_default(&fp);
    if (params) fp = *params;
    Range range("tm_fuse");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    tm_step st{};
    st.kf_id = kf;
    st.n_nbrs = 0;
    st.q_free_off = -1;
    st.nbr_free_off = -1;
    st.mp_begin = 0;
    st.mp_count = mps->n;
    tm_batch_inputs in{};
    in.mps = *mps;
    int32_t po[1] = {0}, fo[2] = {0, 0};
    tm_batch_result r{};
    r.matches = nullptr;
    r.match_cap = 0;
    r.pair_offsets = po;
    r.fuse = out;
    r.fuse_cap = cap;
    r.fuse_offsets = fo;
    tm_status s2 = run_batch_locked(c, &st, 1, &in, sp, fp, &r, pick_stream(c, stream));
    *n_out = r.n_fuse;
    if (n_comparisons) *n_comparisons = r.n_comparisons_fuse;
    return s2;
}

// ------------------------------------------------------------------------- plans

struct tm_plan {
    tm_ctx *ctx = nullptr;
    BatchBuf B;
    std::vector<tm_step> steps;
    std::vector<std::vector<uint64_t>> nbrs;
    int kernels_per_run = 0;
    bool timed_last = false;  // the last run was tm_plan_run_timed
};

extern "C" tm_status tm_debug_bounds(int32_t reset, uint32_t *site, int32_t *enabled) {
    if (!site || !enabled) return fail(TM_ERR_INVALID_ARG, "tm_debug_bounds: null argument");
    bool en = false;
    cudaError_t e = debug_bounds(reset != 0, site, &en);
    *enabled = en ? 1 : 0;
    return e == cudaSuccess ? TM_OK : cuda_fail(e, "bounds status");
}

extern "C" tm_status tm_measure_int_rates(int32_t device, double *popc_per_s, double *lop3_per_s,
                                          double *hamming_per_s) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(TM_ERR_INVALID_ARG, "tm_measure_int_rates: bad device %d", device);
    int prev = 0;
    cudaGetDevice(&prev);
    if ((e = cudaSetDevice(device))) return cuda_fail(e, "cudaSetDevice");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int ctas = 8 * sms, iters = 4096;  // 64 warps per SM
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate[3] = {0.0, 0.0, 0.0};
    tm_status st = TM_OK;
    if ((e = cudaMalloc(&sink, (size_t)ctas * 256 * 4)) || (e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1)))
        st = cuda_fail(e, "tm_measure_int_rates: setup");
    for (int mode = 0; mode < 3 && !st; ++mode) {
        float best = 1e30f;
        for (int r = 0; r < 4 && !st; ++r) {  // the first launch warms up
            if ((e = cudaEventRecord(e0, 0)) || (e = launch_int_rate(mode, ctas, iters, sink, 0)) ||
                (e = cudaEventRecord(e1, 0)) || (e = cudaEventSynchronize(e1))) {
                st = cuda_fail(e, "tm_measure_int_rates: probe");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, ms);
        }
        // operations per launch: mode 0, 1: 8 per round; mode 2: one distance per round
        const double ops = (double)ctas * 256.0 * iters * (mode == 2 ? 1.0 : 8.0);
        rate[mode] = ops / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    if (st) return st;
    if (popc_per_s) *popc_per_s = rate[0];
    if (lop3_per_s) *lop3_per_s = rate[1];
    if (hamming_per_s) *hamming_per_s = rate[2];
    return TM_OK;
}

extern "C" tm_status tm_debug_set(tm_ctx *c, int32_t what, int64_t value) {
    if (!c) return fail(TM_ERR_INVALID_ARG, "tm_debug_set: null context");
    std::lock_guard<std::mutex> lk(c->mu);
    switch (what) {
        case TM_DEBUG_WAIT_LIMIT:
            if (value <= 0) return fail(TM_ERR_INVALID_ARG, "tm_debug_set: wait limit must be > 0");
            c->wait_limit = (long long)value;
            return TM_OK;
        case TM_DEBUG_STARVE_WAITS:
            c->starve = value ? 1u : 0u;
            return TM_OK;
        case TM_DEBUG_SEARCH_THREADS:
            if (value != 0 && value != 256)
                return fail(TM_ERR_INVALID_ARG, "tm_debug_set: search threads must be 0 or 256");
            c->force_threads = (int)value;
            return TM_OK;
        case TM_DEBUG_BRANCH_PRIORITY:
            if (value < -1 || value > 2)
                return fail(TM_ERR_INVALID_ARG, "tm_debug_set: branch priority must be -1, 0, 1 or 2");
            c->branch_prio = (int)value;
            return TM_OK;
        case TM_DEBUG_QUERIES_PER_LANE:
            if (value < 0 || value > 4) return fail(TM_ERR_INVALID_ARG, "tm_debug_set: group form must be 0 .. 4");
            c->force_qpl = (int)value;
            return TM_OK;
        case TM_DEBUG_ENTRY_CAP:
            if (value < 0 || value > kEntryCapMax) return fail(TM_ERR_INVALID_ARG, "tm_debug_set: entry capacity out of range");
            c->entry_cap = value;
            return TM_OK;
        case TM_DEBUG_PERSISTENT:
            if (value < -1 || value > 1) return fail(TM_ERR_INVALID_ARG, "tm_debug_set: persistent must be -1, 0 or 1");
            c->force_persist = (int)value;
            return TM_OK;
        case TM_DEBUG_SPLIT_MIN:
            if (value < -TM_MAX_KP_LIMIT || value > TM_MAX_KP_LIMIT)
                return fail(TM_ERR_INVALID_ARG, "tm_debug_set: split threshold out of range");
            c->split_min = (int)value;
            return TM_OK;
        case TM_DEBUG_L2_PREFETCH:
            if (value < -1 || value > 1) return fail(TM_ERR_INVALID_ARG, "tm_debug_set: L2 prefetch must be -1, 0 or 1");
            c->force_prefetch = (int)value;
            return TM_OK;
        default:
            return fail(TM_ERR_INVALID_ARG, "tm_debug_set: unknown setting %d", (int)what);
    }
}

extern "C" tm_status tm_plan_create(tm_ctx *c, const tm_step *steps, int32_t n_steps,
                                    const tm_batch_inputs *in, const tm_search_params *sp,
                                    const tm_fuse_params *fp, tm_plan **out) {
    if (!c || !out) return fail(TM_ERR_INVALID_ARG, "tm_plan_create: null argument");
    *out = nullptr;
    tm_search_params spd;
    tm_fuse_params fpd;
    tm_search_params_default(&spd);
    tm_fuse_params_default(&fpd);
    if (sp) spd = *sp;
    if (fp) fpd = *fp;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    tm_plan *P = new tm_plan();
    P->ctx = c;
    cudaStream_t s = c->stream;
    tm_status st = prepare_batch(c, P->B, steps, n_steps, in, spd, fpd, s);
    if (!st && spd.mode != TM_MODE_PER_PAIR) {
        if (spd.lanes_per_query) {
            P->B.threads = default_threads(c, P->B);
            P->B.lanes = spd.lanes_per_query;
        } else {
            const char *nt = getenv("TM_NO_TUNE");
            st = tune_batch(c, P->B, steps, s, !(nt && nt[0] == '1'));
            if (!st) {
                c->last_threads = P->B.threads;
                c->last_lanes = P->B.lanes;
                c->last_knobs = P->B.knobs;
                c->last_staged = 1;
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (!st && e) st = cuda_fail(e, "plan upload");
    if (st) {
        drop_new_keyframes(c, P->B, in);
        P->B.release();
        delete P;
        return st;
    }
    if (spd.mode != TM_MODE_PER_PAIR) {
        // capture the launch in two CUDA graphs: kernels only, and the same with events at the
        // stage boundaries (tm_plan_run_timed)
        const int th = P->B.threads, ln = P->B.lanes;
        for (int timed = 0; timed < 2 && !st; ++timed) {
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal)))
                st = cuda_fail(e, "begin capture");
            if (!st) {
                tm_status s1 = enqueue_fused(c, P->B, th, ln, c->capture_stream, timed != 0);
                e = cudaStreamEndCapture(c->capture_stream, &g);
                if (s1) st = s1;
                else if (e) st = cuda_fail(e, "end capture");
            }
            cudaGraphExec_t &x = timed ? P->B.graph_timed : P->B.graph;
            if (!st && (e = cudaGraphInstantiate(&x, g, 0))) st = cuda_fail(e, "graph instantiate");
            if (g) cudaGraphDestroy(g);
        }
        // search (when there are pairs), fuse (when there are map points), copy, ingest (when
        // keyframes enter with the batch)
        // (the entry form's search is three launches: join, evaluation, finalize)
        // (each branch compacts its own records: a copy per part that has items)
        P->kernels_per_run = (P->B.n_search_items ? (P->B.args.qpl == 4 ? 4 : 2) + 1 : 0) +
                             (P->B.n_items > P->B.n_search_items ? 2 : 0) +
                             (P->B.n_new ? 1 : 0) + (P->B.n_search_items && P->B.args.sp.dense_min > 0 ? 1 : 0) +
                             (P->B.n_search_items && P->B.args.triangulate ? 1 : 0);
    } else {
        P->kernels_per_run = 3 * (int)P->B.n_search_items + (P->B.n_new ? 1 : 0) +
                             (P->B.n_search_items && P->B.args.triangulate ? 1 : 0);
        for (int k = 0; k < P->B.n_steps; ++k)
            if (P->B.step_fuse_item[k] != P->B.step_fuse_item[k + 1]) P->kernels_per_run += 2;
        for (int p = 0; P->B.any_fwd && p < P->B.n_pairs; ++p)
            if (P->B.pair_fwd_item[p] != P->B.pair_fwd_item[p + 1]) P->kernels_per_run += 2;
        P->B.lanes = spd.lanes_per_query ? spd.lanes_per_query : 1;
    }
    if (st) {
        cudaStreamSynchronize(c->stream);
        drop_new_keyframes(c, P->B, in);
        P->B.release();
        delete P;
        return st;
    }
    for (int sl : P->B.slots) c->slots[sl].refs++;
    P->steps.assign(steps, steps + n_steps);
    P->nbrs.resize(n_steps);
    for (int k = 0; k < n_steps; ++k) {
        P->nbrs[k].assign(steps[k].nbr_ids, steps[k].nbr_ids + steps[k].n_nbrs);
        P->steps[k].nbr_ids = P->nbrs[k].data();
    }
    *out = P;
    return TM_OK;
}

static tm_status plan_run(tm_plan *P, void *stream, bool timed) {
    Range range(timed ? "tm_plan_run_timed" : "tm_plan_run");
    if (!P) return fail(TM_ERR_INVALID_ARG, "tm_plan_run: null plan");
    tm_ctx *c = P->ctx;
    cudaSetDevice(c->device);
    cudaStream_t s = pick_stream(c, stream);
    cudaGraphExec_t g = timed ? P->B.graph_timed : P->B.graph;
    if (g) {
        cudaError_t e = cudaGraphLaunch(g, s);
        if (e) return cuda_fail(e, "graph launch");
        P->timed_last = timed;
        return TM_OK;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    P->timed_last = false;
    if (P->B.sp.mode == TM_MODE_PER_PAIR) return enqueue_plain(c, P->B, P->B.lanes, s);
    return enqueue_fused(c, P->B, P->B.threads, P->B.lanes, s);
}

extern "C" tm_status tm_plan_run(tm_plan *P, void *stream) { return plan_run(P, stream, false); }

extern "C" tm_status tm_plan_run_timed(tm_plan *P, void *stream) { return plan_run(P, stream, true); }

extern "C" tm_status tm_plan_results(tm_plan *P, tm_batch_result *res, void *stream) {
    if (!P || !res) return fail(TM_ERR_INVALID_ARG, "tm_plan_results: null argument");
    cudaSetDevice(P->ctx->device);
    return fetch_results(P->ctx, P->B, res, pick_stream(P->ctx, stream));
}

extern "C" tm_status tm_plan_info(tm_plan *P, int32_t *threads, int32_t *lanes, int32_t *ctas,
                                  int32_t *kernels) {
    if (!P) return fail(TM_ERR_INVALID_ARG, "tm_plan_info: null plan");
    if (threads) *threads = P->B.threads;
    if (lanes) *lanes = P->B.lanes;
    if (ctas) *ctas = P->B.ctas;
    if (kernels) *kernels = P->kernels_per_run;
    return TM_OK;
}

extern "C" tm_status tm_plan_get_tuning(tm_plan *P, tm_plan_tuning *out) {
    if (!P || !out) return fail(TM_ERR_INVALID_ARG, "tm_plan_get_tuning: null argument");
    const BatchArgs &A = P->B.args;
    const bool fused = P->B.sp.mode != TM_MODE_PER_PAIR;
    out->queries_per_warp = fused ? 32 * (int)(A.qpl >= 3 ? 2 : A.qpl) : 0;
    out->per_lane = fused && A.qpl == 3 ? 1 : 0;
    out->entry_form = fused && A.qpl == 4 ? 1 : 0;
    out->persistent = fused ? (int)A.persist : 0;
    out->l2_prefetch = fused ? (int)A.l2_prefetch : 0;
    out->branch_priority = fused ? (P->ctx->branch_prio >= 0 ? P->ctx->branch_prio : P->B.knobs.bprio) : 0;
    out->dense_min = fused && A.sp.dense_min > 0 ? A.sp.dense_min : 0;
    out->dense_split = out->dense_min > 0 ? (int)A.dsplit : 0;
    out->search_ctas = fused ? P->B.ctas : 0;
    out->tuned = P->B.tuned ? 1 : 0;
    out->search_units = fused ? (int)P->B.n_units : 0;
    return TM_OK;
}

extern "C" tm_status tm_plan_stage_times(tm_plan *P, float *ms) {
    if (!P || !ms) return fail(TM_ERR_INVALID_ARG, "tm_plan_stage_times: null argument");
    for (int k = 0; k < TM_PLAN_STAGES; ++k) ms[k] = 0.0f;
    if (!P->timed_last || !P->B.ev[0]) return TM_OK;
    cudaSetDevice(P->ctx->device);
    cudaError_t e = cudaEventSynchronize(P->B.ev[4]);
    if (e) return cuda_fail(e, "stage events");
    const bool dense = P->B.args.sp.dense_min > 0 && P->B.n_search_items > 0;
    float t[8] = {0};
    for (int k = 1; k < 8; ++k)
        if ((k != 6 || dense) && (e = cudaEventElapsedTime(&t[k], P->B.ev[0], P->B.ev[k])))
            return cuda_fail(e, "stage times");
    ms[0] = t[1] - (dense ? t[6] : t[7]); // search kernel (between the events around it)
    ms[1] = t[2];                         // ingest (from the start)
    ms[2] = t[3] - t[2];                  // fusion (after the ingest)
    ms[3] = t[4] - std::max(t[1], t[3]);  // each branch's offsets + copy, after the later kernel
    ms[4] = dense ? t[6] - t[7] : 0.0f;   // dense node blocks (before the search kernel)
    ms[5] = t[7] - t[5];                  // prep (per-pair constants and eligibility)
    return TM_OK;
}

extern "C" tm_status tm_plan_destroy(tm_plan *P) {
    if (!P) return fail(TM_ERR_INVALID_ARG, "tm_plan_destroy: null plan");
    tm_ctx *c = P->ctx;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        cudaDeviceSynchronize();
        for (int sl : P->B.slots) c->slots[sl].refs--;
    }
    P->B.release();
    delete P;
    return TM_OK;
}
