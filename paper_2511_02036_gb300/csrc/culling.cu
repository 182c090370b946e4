// Host-side map structures of local mapping that stay on the CPU.
//
// Keyframe culling support (Sec. IV-F): the redundancy test of a keyframe counts, for each of
// its map points, how many other keyframes observe the point at the same or a finer scale.
// Instead of walking each map point's observation list, a small array per map point holds the
// number of observations at each pyramid level, updated as observations are added and removed;
// the test then reads a prefix sum of that array.  Host code: the paper keeps this stage on the
// CPU (its observation data change every iteration).
//
// Fuse-apply (Sec. IV-D): the fusion search runs in parallel on the GPU against one state of
// the map and only lists candidate duplicate pairs; merging them is deferred to a sequential
// stage, tm_map_fuse_apply below, which applies the candidates in order against the map as it
// stands, so that the outcome is that of the sequential loop.

#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "runtime.h"
#include "tm.h"

// Map points of a keyframe observed at level L count as redundant when at least th_obs other
// keyframes observe them at a level <= L + 1 (the keyframe's own observation is in cnt).
template <typename C>
static bool point_redundant(const C *cnt, int level, int32_t th_obs) {
    const int top = level + 1 < TM_LEVELS ? level + 1 : TM_LEVELS - 1;
    int64_t seen = 0;
    for (int l = 0; l <= top; ++l) seen += cnt[l];
    return seen - 1 >= th_obs;
}

struct tm_obs_counter {
    int32_t max_mps = 0;
    std::vector<uint16_t> counts;  // [max_mps][TM_LEVELS]
    std::mutex mu;
};

using namespace tmap;

static tm_status check_obs(const tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level) {
    if (!c || n < 0 || (n > 0 && (!mp || !level))) return fail(TM_ERR_INVALID_ARG, "tm_obs: bad arguments");
    for (int32_t k = 0; k < n; ++k) {
        if (mp[k] < 0 || mp[k] >= c->max_mps)
            return fail(TM_ERR_INVALID_ARG, "tm_obs: map point %d outside 0..%d", mp[k], c->max_mps - 1);
        if (level[k] >= TM_LEVELS) return fail(TM_ERR_INVALID_ARG, "tm_obs: level %d >= %d", level[k], TM_LEVELS);
    }
    return TM_OK;
}

extern "C" tm_status tm_obs_create(int32_t max_mps, tm_obs_counter **out) {
    if (!out || max_mps <= 0) return fail(TM_ERR_INVALID_ARG, "tm_obs_create: bad arguments");
    tm_obs_counter *c = new (std::nothrow) tm_obs_counter;
    if (!c) return fail(TM_ERR_NO_MEMORY, "tm_obs_create: out of host memory");
    try {
        c->counts.assign((size_t)max_mps * TM_LEVELS, 0);
    } catch (...) {
        delete c;
        return fail(TM_ERR_NO_MEMORY, "tm_obs_create: out of host memory");
    }
    c->max_mps = max_mps;
    *out = c;
    return TM_OK;
}

extern "C" tm_status tm_obs_destroy(tm_obs_counter *c) {
    if (!c) return fail(TM_ERR_INVALID_ARG, "tm_obs_destroy: null");
    delete c;
    return TM_OK;
}

extern "C" tm_status tm_obs_add(tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level) {
    tm_status st = check_obs(c, n, mp, level);
    if (st) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    for (int32_t k = 0; k < n; ++k)
        if (c->counts[(size_t)mp[k] * TM_LEVELS + level[k]] == UINT16_MAX)
            return fail(TM_ERR_CAPACITY, "tm_obs_add: more than 65535 observations of map point %d at level %d "
                        "(the earlier entries of this call were added)", mp[k], level[k]);
        else
            ++c->counts[(size_t)mp[k] * TM_LEVELS + level[k]];
    return TM_OK;
}

extern "C" tm_status tm_obs_remove(tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level) {
    tm_status st = check_obs(c, n, mp, level);
    if (st) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    // all or nothing: every removal must have an observation to remove (counted per counter,
    // so that a counter named several times needs as many observations)
    std::unordered_map<size_t, uint32_t> need;
    for (int32_t k = 0; k < n; ++k) {
        const size_t e = (size_t)mp[k] * TM_LEVELS + level[k];
        if (c->counts[e] <= need[e]++)
            return fail(TM_ERR_NOT_FOUND, "tm_obs_remove: no observation of map point %d at level %d to remove",
                        mp[k], level[k]);
    }
    for (int32_t k = 0; k < n; ++k) --c->counts[(size_t)mp[k] * TM_LEVELS + level[k]];
    return TM_OK;
}

extern "C" tm_status tm_obs_redundant(tm_obs_counter *c, int32_t n, const int32_t *mp, const uint8_t *level,
                                      int32_t th_obs, float ratio, int32_t *n_redundant,
                                      int32_t *is_redundant) {
    tm_status st = check_obs(c, n, mp, level);
    if (st) return st;
    if (!n_redundant || !is_redundant || th_obs < 0 || !(ratio >= 0.0f))
        return fail(TM_ERR_INVALID_ARG, "tm_obs_redundant: bad arguments");
    std::lock_guard<std::mutex> lk(c->mu);
    int32_t red = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (point_redundant(&c->counts[(size_t)mp[k] * TM_LEVELS], level[k], th_obs)) ++red;
    }
    *n_redundant = red;
    *is_redundant = (float)red > ratio * (float)n ? 1 : 0;
    return TM_OK;
}

// ---------------------------------------------------------------------------- fuse-apply

namespace {

struct MapKeyframe {
    std::vector<int32_t> kp_mp;  // keypoint -> map point, -1 none
    std::vector<uint8_t> level;  // keypoint -> pyramid level
};

enum : uint8_t { MP_NONE = 0, MP_LIVE = 1, MP_REPLACED = 2 };

struct MapPoint {
    uint8_t state = MP_NONE;
    int32_t replaced_by = -1;
    std::vector<std::pair<uint64_t, int32_t>> obs;  // (keyframe, keypoint), in insertion order
};

}  // namespace

struct tm_map {
    int32_t max_mps = 0;
    std::unordered_map<uint64_t, MapKeyframe> kfs;
    std::vector<MapPoint> mps;
    std::vector<uint32_t> counts;  // [max_mps][TM_LEVELS] observations per level
    std::mutex mu;

    int32_t observed_at(int32_t p, uint64_t kf) const {
        for (const auto &o : mps[p].obs)
            if (o.first == kf) return o.second;
        return -1;
    }
    uint32_t &count(int32_t p, const MapKeyframe &k, int32_t kp) {
        return counts[(size_t)p * TM_LEVELS + k.level[kp]];
    }
    void observe(int32_t p, uint64_t kf_id, MapKeyframe &k, int32_t kp) {
        mps[p].state = MP_LIVE;
        mps[p].obs.emplace_back(kf_id, kp);
        k.kp_mp[kp] = p;
        ++count(p, k, kp);
    }
    // Point a is replaced by point b: a's observations move to b, except in keyframes that
    // already observe b, where the keypoint loses its map point.
    void replace(int32_t a, int32_t b) {
        std::vector<std::pair<uint64_t, int32_t>> moved;
        moved.swap(mps[a].obs);
        for (const auto &o : moved) {
            MapKeyframe &k = kfs.at(o.first);
            --count(a, k, o.second);
            if (observed_at(b, o.first) >= 0) {
                k.kp_mp[o.second] = -1;
            } else {
                mps[b].obs.push_back(o);
                k.kp_mp[o.second] = b;
                ++count(b, k, o.second);
            }
        }
        mps[a].state = MP_REPLACED;
        mps[a].replaced_by = b;
    }
};

extern "C" tm_status tm_map_create(int32_t max_mps, tm_map **out) {
    if (!out || max_mps <= 0) return fail(TM_ERR_INVALID_ARG, "tm_map_create: bad arguments");
    tm_map *m = new (std::nothrow) tm_map;
    if (!m) return fail(TM_ERR_NO_MEMORY, "tm_map_create: out of host memory");
    try {
        m->mps.resize((size_t)max_mps);
        m->counts.assign((size_t)max_mps * TM_LEVELS, 0);
    } catch (...) {
        delete m;
        return fail(TM_ERR_NO_MEMORY, "tm_map_create: out of host memory");
    }
    m->max_mps = max_mps;
    *out = m;
    return TM_OK;
}

extern "C" tm_status tm_map_destroy(tm_map *m) {
    if (!m) return fail(TM_ERR_INVALID_ARG, "tm_map_destroy: null");
    delete m;
    return TM_OK;
}

extern "C" tm_status tm_map_add_keyframe(tm_map *m, uint64_t kf_id, int32_t n_kp, const uint8_t *level) {
    if (!m || n_kp < 0) return fail(TM_ERR_INVALID_ARG, "tm_map_add_keyframe: bad arguments");
    if (level)
        for (int32_t i = 0; i < n_kp; ++i)
            if (level[i] >= TM_LEVELS)
                return fail(TM_ERR_INVALID_ARG, "tm_map_add_keyframe: level %d >= %d", level[i], TM_LEVELS);
    std::lock_guard<std::mutex> lk(m->mu);
    if (m->kfs.count(kf_id)) return fail(TM_ERR_EXISTS, "tm_map_add_keyframe: keyframe %llu exists",
                                         (unsigned long long)kf_id);
    try {
        MapKeyframe k;
        k.kp_mp.assign((size_t)n_kp, -1);
        if (level) k.level.assign(level, level + n_kp);
        else k.level.assign((size_t)n_kp, 0);
        m->kfs.emplace(kf_id, std::move(k));
    } catch (...) {
        return fail(TM_ERR_NO_MEMORY, "tm_map_add_keyframe: out of host memory");
    }
    return TM_OK;
}

extern "C" tm_status tm_map_remove_keyframe(tm_map *m, uint64_t kf_id) {
    if (!m) return fail(TM_ERR_INVALID_ARG, "tm_map_remove_keyframe: null");
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->kfs.find(kf_id);
    if (it == m->kfs.end())
        return fail(TM_ERR_NOT_FOUND, "tm_map_remove_keyframe: keyframe %llu not in the map",
                    (unsigned long long)kf_id);
    MapKeyframe &k = it->second;
    for (int32_t i = 0; i < (int32_t)k.kp_mp.size(); ++i) {
        const int32_t p = k.kp_mp[i];
        if (p < 0) continue;
        auto &obs = m->mps[p].obs;
        for (size_t q = 0; q < obs.size(); ++q)
            if (obs[q].first == kf_id) {
                obs.erase(obs.begin() + (ptrdiff_t)q);
                break;
            }
        --m->count(p, k, i);
    }
    m->kfs.erase(it);
    return TM_OK;
}

extern "C" tm_status tm_map_add_observations(tm_map *m, uint64_t kf_id, int32_t n, const int32_t *kp,
                                             const int32_t *mp) {
    if (!m || n < 0 || (n > 0 && (!kp || !mp)))
        return fail(TM_ERR_INVALID_ARG, "tm_map_add_observations: bad arguments");
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->kfs.find(kf_id);
    if (it == m->kfs.end())
        return fail(TM_ERR_NOT_FOUND, "tm_map_add_observations: keyframe %llu not in the map",
                    (unsigned long long)kf_id);
    MapKeyframe &k = it->second;
    const int32_t n_kp = (int32_t)k.kp_mp.size();
    std::unordered_map<int32_t, int32_t> seen_kp, seen_mp;  // first entry naming each
    for (int32_t e = 0; e < n; ++e) {
        if (kp[e] < 0 || kp[e] >= n_kp || mp[e] < 0 || mp[e] >= m->max_mps)
            return fail(TM_ERR_INVALID_ARG, "tm_map_add_observations: entry %d (keypoint %d, map point %d) "
                        "out of range", e, kp[e], mp[e]);
        if (k.kp_mp[kp[e]] >= 0)
            return fail(TM_ERR_INVALID_ARG, "tm_map_add_observations: keypoint %d already has map point %d",
                        kp[e], k.kp_mp[kp[e]]);
        if (m->mps[mp[e]].state == MP_REPLACED)
            return fail(TM_ERR_INVALID_ARG, "tm_map_add_observations: map point %d was replaced", mp[e]);
        if (m->observed_at(mp[e], kf_id) >= 0)
            return fail(TM_ERR_INVALID_ARG, "tm_map_add_observations: keyframe already observes map point %d",
                        mp[e]);
        const auto a = seen_kp.emplace(kp[e], e), b = seen_mp.emplace(mp[e], e);
        if (!a.second || !b.second)
            return fail(TM_ERR_INVALID_ARG, "tm_map_add_observations: entries %d and %d share a keypoint "
                        "or a map point", !a.second ? a.first->second : b.first->second, e);
    }
    for (int32_t e = 0; e < n; ++e) m->observe(mp[e], kf_id, k, kp[e]);
    return TM_OK;
}

extern "C" tm_status tm_map_fuse_apply(tm_map *m, uint64_t kf_id, int32_t n, const tm_fuse_match *cand,
                                       const int32_t *mp_ids, int32_t n_ids, tm_fuse_apply_stats *stats) {
    if (!m || n < 0 || (n > 0 && !cand) || (mp_ids && n_ids < 0))
        return fail(TM_ERR_INVALID_ARG, "tm_map_fuse_apply: bad arguments");
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->kfs.find(kf_id);
    if (it == m->kfs.end())
        return fail(TM_ERR_NOT_FOUND, "tm_map_fuse_apply: keyframe %llu not in the map",
                    (unsigned long long)kf_id);
    MapKeyframe &k = it->second;
    const int32_t n_kp = (int32_t)k.kp_mp.size();
    for (int32_t e = 0; e < n; ++e) {
        const int32_t j = cand[e].kp_idx, b = cand[e].mp_idx;
        if (j < 0 || j >= n_kp)
            return fail(TM_ERR_INVALID_ARG, "tm_map_fuse_apply: candidate %d: keypoint %d outside 0..%d", e, j,
                        n_kp - 1);
        if (mp_ids && (b < 0 || b >= n_ids))
            return fail(TM_ERR_INVALID_ARG, "tm_map_fuse_apply: candidate %d: batch index %d outside 0..%d", e,
                        b, n_ids - 1);
        const int32_t p = mp_ids ? mp_ids[b] : b;
        if (p < 0 || p >= m->max_mps || m->mps[p].state == MP_NONE)
            return fail(TM_ERR_INVALID_ARG, "tm_map_fuse_apply: candidate %d: map point %d does not exist", e, p);
    }
    Range range("tm_map_fuse_apply");
    tm_fuse_apply_stats st = {0, 0, 0, 0, 0};
    for (int32_t e = 0; e < n; ++e) {
        const int32_t j = cand[e].kp_idx;
        const int32_t mp = mp_ids ? mp_ids[cand[e].mp_idx] : cand[e].mp_idx;
        if (m->mps[mp].state != MP_LIVE) {
            ++st.skipped_dead;
            continue;
        }
        if (m->observed_at(mp, kf_id) >= 0) {
            ++st.skipped_observed;
            continue;
        }
        const int32_t p = k.kp_mp[j];
        if (p < 0) {
            m->observe(mp, kf_id, k, j);
            ++st.added;
        } else if (m->mps[p].obs.size() > m->mps[mp].obs.size()) {
            m->replace(mp, p);
            ++st.merged_into_existing;
        } else {
            m->replace(p, mp);
            ++st.replaced_existing;
        }
    }
    if (stats) *stats = st;
    return TM_OK;
}

extern "C" tm_status tm_map_keyframe_points(tm_map *m, uint64_t kf_id, int32_t n_kp, int32_t *out) {
    if (!m || n_kp < 0 || (n_kp > 0 && !out)) return fail(TM_ERR_INVALID_ARG, "tm_map_keyframe_points: bad arguments");
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->kfs.find(kf_id);
    if (it == m->kfs.end())
        return fail(TM_ERR_NOT_FOUND, "tm_map_keyframe_points: keyframe %llu not in the map",
                    (unsigned long long)kf_id);
    if ((size_t)n_kp != it->second.kp_mp.size())
        return fail(TM_ERR_INVALID_ARG, "tm_map_keyframe_points: n_kp %d, keyframe has %zu", n_kp,
                    it->second.kp_mp.size());
    if (n_kp) std::memcpy(out, it->second.kp_mp.data(), sizeof(int32_t) * (size_t)n_kp);
    return TM_OK;
}

extern "C" tm_status tm_map_point_info(tm_map *m, int32_t n, const int32_t *mp, int32_t *live, int32_t *current,
                                       int32_t *n_obs) {
    if (!m || n < 0 || (n > 0 && !mp)) return fail(TM_ERR_INVALID_ARG, "tm_map_point_info: bad arguments");
    for (int32_t e = 0; e < n; ++e)
        if (mp[e] < 0 || mp[e] >= m->max_mps)
            return fail(TM_ERR_INVALID_ARG, "tm_map_point_info: map point %d outside 0..%d", mp[e], m->max_mps - 1);
    std::lock_guard<std::mutex> lk(m->mu);
    for (int32_t e = 0; e < n; ++e) {
        const MapPoint &p = m->mps[mp[e]];
        int32_t cur = p.state == MP_NONE ? -1 : mp[e];
        // a replacement chain is acyclic (a replaced point never becomes live again), so this ends
        while (cur >= 0 && m->mps[cur].state == MP_REPLACED) cur = m->mps[cur].replaced_by;
        if (live) live[e] = p.state == MP_LIVE ? 1 : p.state == MP_REPLACED ? 0 : -1;
        if (current) current[e] = cur;
        if (n_obs) n_obs[e] = (int32_t)p.obs.size();
    }
    return TM_OK;
}

extern "C" tm_status tm_map_redundant(tm_map *m, uint64_t kf_id, int32_t th_obs, float ratio, int32_t *n_redundant,
                                      int32_t *is_redundant) {
    if (!m || !n_redundant || !is_redundant || th_obs < 0 || !(ratio >= 0.0f))
        return fail(TM_ERR_INVALID_ARG, "tm_map_redundant: bad arguments");
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->kfs.find(kf_id);
    if (it == m->kfs.end())
        return fail(TM_ERR_NOT_FOUND, "tm_map_redundant: keyframe %llu not in the map", (unsigned long long)kf_id);
    const MapKeyframe &k = it->second;
    int32_t n = 0, red = 0;
    for (size_t i = 0; i < k.kp_mp.size(); ++i) {
        const int32_t p = k.kp_mp[i];
        if (p < 0) continue;
        ++n;
        if (point_redundant(&m->counts[(size_t)p * TM_LEVELS], k.level[i], th_obs)) ++red;
    }
    *n_redundant = red;
    *is_redundant = (float)red > ratio * (float)n ? 1 : 0;
    return TM_OK;
}
