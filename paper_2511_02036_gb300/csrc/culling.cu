// Keyframe culling support (Sec. IV-F): the redundancy test of a keyframe counts, for each of
// its map points, how many other keyframes observe the point at the same or a finer scale.
// Instead of walking each map point's observation list, a small array per map point holds the
// number of observations at each pyramid level, updated as observations are added and removed;
// the test then reads a prefix sum of that array.  Host code: the paper keeps this stage on the
// CPU (its observation data change every iteration).

#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "runtime.h"
#include "tm.h"

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
    // all or nothing: every removal must have an observation to remove
    std::vector<uint32_t> need;
    for (int32_t k = 0; k < n; ++k) {
        const size_t e = (size_t)mp[k] * TM_LEVELS + level[k];
        uint32_t earlier = 0;
        for (int32_t q = 0; q < k; ++q)
            if (mp[q] == mp[k] && level[q] == level[k]) ++earlier;
        if (c->counts[e] <= earlier)
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
        const uint16_t *cnt = &c->counts[(size_t)mp[k] * TM_LEVELS];
        // observations at level <= own level + 1, the keyframe's own among them
        const int top = level[k] + 1 < TM_LEVELS ? level[k] + 1 : TM_LEVELS - 1;
        int32_t seen = 0;
        for (int l = 0; l <= top; ++l) seen += cnt[l];
        if (seen - 1 >= th_obs) ++red;
    }
    *n_redundant = red;
    *is_redundant = (float)red > ratio * (float)n ? 1 : 0;
    return TM_OK;
}
