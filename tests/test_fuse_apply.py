"""Fuse-apply, the sequential stage after the parallel fusion search (Sec. IV-D): the library's
host-side map (tm_map_*) against the oracle's plain-dictionary twin, both against a case worked
by hand (tests/golden/fuse_apply_worked.json), and the oracle against the map's consistency
invariants.  Host code only: no GPU is needed."""

import json
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "fuse_apply_worked.json")))
IDS = {"A": 11, "B": 12, "C": 13, "T": 14}


@pytest.fixture(scope="module")
def tm():
    import __graft_entry__ as g
    g.build()
    import paper_2511_02036_gb300 as tm
    return tm


def oracle_map(g):
    fm = O.FuseMap()
    for k, lv in g["keyframes"].items():
        fm.add_keyframe(k, len(lv), lv)
    for m, obs in g["observations"].items():
        for k, j in obs:
            fm.observe(k, j, int(m))
    return fm


def library_map(tm, g, max_mps=64):
    mp = tm.Map(max_mps)
    for k, lv in g["keyframes"].items():
        mp.add_keyframe(IDS[k], len(lv), lv)
    per_kf = {}
    for m, obs in g["observations"].items():
        for k, j in obs:
            per_kf.setdefault(k, []).append((j, int(m)))
    for k, lst in per_kf.items():
        mp.add_observations(IDS[k], [j for j, _ in lst], [m for _, m in lst])
    return mp


def check_consistent(fm):
    """The map's invariants: keypoint -> point and point -> (keyframe, keypoint) agree both ways,
    no point is both live and replaced, and every replacement chain ends at a live point."""
    links = 0
    for k, row in fm.kp.items():
        for j, m in enumerate(row):
            if m is not None:
                links += 1
                assert fm.obs[m][k] == j
    assert links == sum(len(o) for o in fm.obs.values())
    for m, o in fm.obs.items():
        assert m not in fm.replaced
        for k, j in o.items():
            assert fm.kp[k][j] == m
    for m in fm.replaced:
        assert fm.current(m) in fm.obs
    return links


def test_oracle_worked_case():
    g, exp = GOLD, GOLD["expected"]
    fm = oracle_map(g)
    assert fm.fuse(g["target"], [tuple(c) for c in g["candidates"]]) == exp["stats"]
    for k, row in exp["keyframes"].items():
        assert fm.kp[k] == row
    for m, c in exp["current"].items():
        assert fm.current(int(m)) == c
    assert {m: len(o) for m, o in fm.obs.items()} == {int(m): n for m, n in exp["n_obs"].items()}
    for r in exp["redundant"]:
        assert O.culling_redundant(fm.observations(), r["kf"], r["th_obs"], r["ratio"]) == \
            (r["n_redundant"], r["redundant"]), r
    check_consistent(fm)


@pytest.mark.parametrize("indexed", [False, True])
def test_library_worked_case(tm, indexed):
    g, exp = GOLD, GOLD["expected"]
    with library_map(tm, g) as mp:
        cands = np.array([[m, j, 0] for m, j in g["candidates"]], np.int32)
        ids = None
        if indexed:  # candidates as a batch result: mp_idx indexes the batch's id table
            ids = np.array([0, 10, 9, 8, 7, 6, 5, 4, 3, 2, 1], np.int32)
            cands[:, 0] = 11 - cands[:, 0]
        assert mp.fuse_apply(IDS[g["target"]], cands, ids) == exp["stats"]
        for k, row in exp["keyframes"].items():
            np.testing.assert_array_equal(mp.keyframe_points(IDS[k], len(row)),
                                          [-1 if x is None else x for x in row])
        pts = list(range(0, 12))
        live, cur, nobs = mp.point_info(pts)
        for m in pts:
            e = exp["current"].get(str(m))
            assert cur[m] == (-1 if e is None else e)
            assert live[m] == (-1 if e is None else int(e == m))
            assert nobs[m] == exp["n_obs"].get(str(m), 0)
        for r in exp["redundant"]:
            assert mp.redundant(IDS[r["kf"]], r["th_obs"], r["ratio"]) == (r["n_redundant"], r["redundant"]), r


def random_map(rng, n_kf=10, n_mp=300):
    fm = O.FuseMap()
    kfs = {}
    for k in range(n_kf):
        n = int(rng.integers(15, 50))
        kfs[k] = rng.integers(0, 8, n).astype(np.uint8)
        fm.add_keyframe(k, n, kfs[k])
    obs = {k: [] for k in kfs}
    for m in range(n_mp):
        for k in rng.choice(n_kf, size=int(rng.integers(1, 5)), replace=False):
            k = int(k)
            free = [j for j, x in enumerate(fm.kp[k]) if x is None]
            if free:
                j = int(rng.choice(free))
                fm.observe(k, j, m)
                obs[k].append((j, m))
    return fm, kfs, obs


def compare(mp, fm, kfs, n_ids):
    for k, lv in kfs.items():
        np.testing.assert_array_equal(mp.keyframe_points(k, len(lv)),
                                      [-1 if x is None else x for x in fm.kp[k]])
    live, cur, nobs = mp.point_info(np.arange(n_ids))
    for m in range(n_ids):
        ex = 1 if m in fm.obs else 0 if m in fm.replaced else -1
        assert live[m] == ex
        c = fm.current(m)
        assert cur[m] == (-1 if c is None else c)
        assert nobs[m] == len(fm.obs.get(m, {}))
    ob = fm.observations()
    for k in kfs:
        for th, ratio in ((1, 0.5), (2, 0.9), (3, 0.3)):
            assert mp.redundant(k, th, ratio) == O.culling_redundant(ob, k, th, ratio), (k, th, ratio)


@pytest.mark.parametrize("seed", range(4))
def test_library_matches_oracle_random(tm, seed):
    """Random maps and candidate lists (dead points, already-observed targets, empty and held
    keypoints, replacement chains), keyframes culled and added between rounds."""
    rng = np.random.default_rng(7100 + seed)
    n_mp = 300
    fm, kfs, obs = random_map(rng, n_mp=n_mp)
    next_mp, next_kf = n_mp, len(kfs)
    with tm.Map(1000) as mp:
        for k, lv in kfs.items():
            mp.add_keyframe(k, len(lv), lv)
            if obs[k]:
                mp.add_observations(k, [j for j, _ in obs[k]], [m for _, m in obs[k]])
        compare(mp, fm, kfs, next_mp)
        totals = dict(added=0, merged_into_existing=0, replaced_existing=0, skipped_dead=0, skipped_observed=0)
        for rnd in range(40):
            k = int(rng.choice(sorted(kfs)))
            existed = sorted(set(fm.obs) | set(fm.replaced))
            n = int(rng.integers(0, 40))
            cm = rng.choice(existed, size=n) if n else np.zeros(0, np.int64)
            cj = rng.integers(0, len(kfs[k]), n)
            links_before = check_consistent(fm)
            est = fm.fuse(k, list(zip(cm.tolist(), cj.tolist())))
            assert check_consistent(fm) <= links_before + est["added"]
            if rnd % 2:
                ids = rng.permutation(next_mp).astype(np.int32)
                inv = np.argsort(ids)
                c = np.stack([inv[cm], cj, np.zeros(n, np.int64)], 1) if n else np.zeros((0, 3))
                got = mp.fuse_apply(k, c, ids)
            else:
                c = np.stack([cm, cj, np.zeros(n, np.int64)], 1) if n else np.zeros((0, 3))
                got = mp.fuse_apply(k, c)
            assert got == est
            for f in totals:
                totals[f] += est[f]
            if rnd % 10 == 9:  # cull a keyframe, add one with new points and some existing ones
                gone = int(rng.choice(sorted(kfs)))
                fm.remove_keyframe(gone)
                mp.remove_keyframe(gone)
                del kfs[gone]
                nk = next_kf
                next_kf += 1
                kfs[nk] = rng.integers(0, 8, 30).astype(np.uint8)
                fm.add_keyframe(nk, 30, kfs[nk])
                mp.add_keyframe(nk, 30, kfs[nk])
                live = sorted(fm.obs)
                pts = [int(x) for x in rng.choice(live, size=10, replace=False)] + list(range(next_mp, next_mp + 10))
                next_mp += 10
                js = [int(x) for x in rng.permutation(30)[:20]]
                for j, m in zip(js, pts):
                    fm.observe(nk, j, m)
                mp.add_observations(nk, js, pts)
            compare(mp, fm, kfs, next_mp)
        # the random lists exercise every branch
        assert all(v > 0 for v in totals.values()), totals


def test_errors_leave_the_map_unchanged(tm):
    g = GOLD
    with library_map(tm, g) as mp:
        def state():
            return [mp.keyframe_points(IDS[k], len(r)).tolist() for k, r in g["keyframes"].items()] + \
                [x.tolist() for x in mp.point_info(np.arange(12))]
        s0 = state()
        T = IDS["T"]
        bad = [
            (lambda: mp.fuse_apply(T, [[2, 3, 0], [5, 2, 0], [1, 5, 0]]), tm.TM_ERR_INVALID_ARG),  # keypoint 5 of 5
            (lambda: mp.fuse_apply(T, [[2, 3, 0], [20, 2, 0]]), tm.TM_ERR_INVALID_ARG),           # point never existed
            (lambda: mp.fuse_apply(T, [[2, 3, 0], [64, 2, 0]]), tm.TM_ERR_INVALID_ARG),           # beyond max_mps
            (lambda: mp.fuse_apply(T, [[0, 3, 0], [3, 2, 0]], np.array([2, 3, 4])), tm.TM_ERR_INVALID_ARG),  # index 3 of 3
            (lambda: mp.fuse_apply(99, [[2, 3, 0]]), tm.TM_ERR_NOT_FOUND),
            (lambda: mp.add_observations(T, [3, 0], [20, 21]), tm.TM_ERR_INVALID_ARG),            # T0 holds a point
            (lambda: mp.add_observations(T, [3], [4]), tm.TM_ERR_INVALID_ARG),                    # T observes 4
            (lambda: mp.add_observations(IDS["A"], [4, 4], [20, 21]), tm.TM_ERR_INVALID_ARG),     # keypoint twice
            (lambda: mp.add_observations(IDS["A"], [4], [64]), tm.TM_ERR_INVALID_ARG),
            (lambda: mp.add_keyframe(T, 3), tm.TM_ERR_EXISTS),
            (lambda: mp.add_keyframe(50, 2, [0, 8]), tm.TM_ERR_INVALID_ARG),
            (lambda: mp.keyframe_points(T, 4), tm.TM_ERR_INVALID_ARG),
            (lambda: mp.remove_keyframe(50), tm.TM_ERR_NOT_FOUND),
            (lambda: mp.redundant(50), tm.TM_ERR_NOT_FOUND),
        ]
        for f, status in bad:
            with pytest.raises(tm.TMError) as e:
                f()
            assert e.value.status == status
            assert state() == s0
        # a replaced point cannot be observed again
        mp.fuse_apply(T, [[1, 1, 0]])               # 1 merged into 4
        with pytest.raises(tm.TMError) as e:
            mp.add_observations(IDS["C"], [4], [1])
        assert e.value.status == tm.TM_ERR_INVALID_ARG
        assert mp.fuse_apply(T, np.zeros((0, 3), np.int32)) == dict(
            added=0, merged_into_existing=0, replaced_existing=0, skipped_dead=0, skipped_observed=0)


def test_add_observations_all_or_nothing(tm):
    with tm.Map(100) as mp:
        mp.add_keyframe(1, 4)
        mp.add_keyframe(2, 4)
        for kp, pts in (([0, 1], [20, 20]),      # one point at two keypoints of a keyframe
                        ([0, 1, 0], [5, 6, 7]),  # one keypoint twice
                        ([0, 4], [5, 6])):       # keypoint out of range
            with pytest.raises(tm.TMError) as e:
                mp.add_observations(1, kp, pts)
            assert e.value.status == tm.TM_ERR_INVALID_ARG
            np.testing.assert_array_equal(mp.keyframe_points(1, 4), [-1] * 4)
            assert mp.point_info([5, 6, 7, 20])[0].tolist() == [-1] * 4
        mp.add_observations(1, [3, 0], [20, 21])
        mp.add_observations(2, [0], [20])
        np.testing.assert_array_equal(mp.keyframe_points(1, 4), [21, -1, -1, 20])
        assert mp.point_info([20, 21])[2].tolist() == [2, 1]
        mp.remove_keyframe(1)                        # culling erases its observations
        assert mp.point_info([20, 21])[2].tolist() == [1, 0]
        assert mp.point_info([20, 21])[0].tolist() == [1, 1]  # points stay live
        with pytest.raises(tm.TMError):
            mp.keyframe_points(1, 4)
