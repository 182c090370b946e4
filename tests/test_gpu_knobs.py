"""Parity under every launch choice the autotuner can make: queries per warp group (32 or
64), the persistent work-queue search, the L2 prefetch of a pair's descriptors, the branch
priority, and the dense-block split.  Each choice is forced through tm_debug_set on a fresh
context; the fused batch's results must equal the oracle's bit-exactly whatever it is, and
tm_plan_get_tuning must report the choice in effect."""

import itertools

import numpy as np
import pytest

import oracle as O
from gen import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    import __graft_entry__ as g
    g.build()
    import paper_2511_02036_gb300 as tm
    return tm


def osp(sp):
    return O.SearchParams(sp.hamming_max, sp.ratio_num, sp.ratio_den, sp.epi_chi2, sp.epipolar,
                          sp.resolve, sp.rot_filter, sp.epipole_px, sp.rot_mode)


def steps_of(w):
    return [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                 mps=s.get("mps")) for s in w["steps"]]


def expected(w, sp=None):
    pairs, fuses, cs, cf = [], [], 0, 0
    for st in w["steps"]:
        r, c = O.search_step(w["cam"], w["frames"], st, osp(sp) if sp is not None else None)
        pairs.extend(r)
        cs += c
        f, c2 = O.fuse_step(w["cam"], w["frames"], st)
        fuses.append(f)
        cf += c2
    return pairs, fuses, cs, cf


def assert_same(res, exp):
    pairs, fuses, cs, cf = exp
    assert len(res.pairs) == len(pairs) and len(res.fuses) == len(fuses)
    for g, e in zip(res.pairs, pairs):
        np.testing.assert_array_equal(g, e)
    for g, e in zip(res.fuses, fuses):
        np.testing.assert_array_equal(g, e)
    assert res.n_comparisons_search == cs
    assert res.n_comparisons_fuse == cf


def load_all(ctx, w):
    ids = sorted(set(i for s in w["steps"] for i in [s["q"]] + s["nbrs"]))
    ctx.add_keyframes(ids, [w["frames"][i] for i in ids])


@pytest.fixture(scope="module")
def batch():
    # several tiles of queries per pair and a ragged last group (600..2000 keypoints)
    w = W.make_cfg2(seed=2200, n_steps=5)
    return w, expected(w)


def force(tm, ctx, qpl=None, persist=None, prefetch=None, bprio=None):
    from paper_2511_02036_gb300 import _lib as L
    if qpl is not None:
        ctx.debug_set(L.TM_DEBUG_QUERIES_PER_LANE, qpl)
    if persist is not None:
        ctx.debug_set(L.TM_DEBUG_PERSISTENT, persist)
    if prefetch is not None:
        ctx.debug_set(L.TM_DEBUG_L2_PREFETCH, prefetch)
    if bprio is not None:
        ctx.debug_set(L.TM_DEBUG_BRANCH_PRIORITY, bprio)


@pytest.mark.parametrize("qpl,persist,prefetch", list(itertools.product((1, 2), (0, 1), (0, 1))) +
                         [(3, 0, 0), (3, 0, 1), (4, 0, 0)])
def test_search_knobs_match_oracle(tm, batch, qpl, persist, prefetch):
    from paper_2511_02036_gb300 import _lib as L
    w, exp = batch
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        ctx.debug_set(L.TM_DEBUG_SPLIT_MIN, 0)  # (split pairs have no persistent instance)
        force(tm, ctx, qpl=qpl, persist=persist, prefetch=prefetch)
        with ctx.plan(steps_of(w)) as plan:
            t = plan.tuning()
            assert t["queries_per_warp"] == 32 * min(qpl, 2) and t["per_lane"] == (qpl == 3)
            assert t["entry_form"] == (qpl == 4)
            assert t["persistent"] == persist and t["l2_prefetch"] == prefetch
            if persist:
                assert 1 <= t["search_ctas"] <= t["search_units"]
            for _ in range(2):  # the replay resets the persistent work counter
                plan.run()
                assert_same(plan.results(), exp)
        # the one-shot batch takes the same forced choices
        assert_same(ctx.batch_run(steps_of(w)), exp)


@pytest.mark.parametrize("bprio", [0, 1, 2])
def test_branch_priority_matches_oracle(tm, batch, bprio):
    w, exp = batch
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        force(tm, ctx, bprio=bprio)
        with ctx.plan(steps_of(w)) as plan:
            assert plan.tuning()["branch_priority"] == bprio
            plan.run()
            assert_same(plan.results(), exp)


@pytest.mark.parametrize("qpl", [1, 2, 3, 4])
def test_variant_gates_ignore_persistent(tm, qpl):
    """With the epipole rejection on, the search takes its general instance (rounds, 64-query
    groups): the persistent and per-lane requests are set aside (reported as 0), the results
    still equal the oracle's."""
    w = W.make_cfg2(seed=2201, n_steps=3)
    sp = tm.SearchParams(epipole_px=12.0)
    exp = expected(w, sp)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        force(tm, ctx, qpl=qpl, persist=1)
        with ctx.plan(steps_of(w), sp=sp) as plan:
            t = plan.tuning()
            assert t["persistent"] == 0 and t["per_lane"] == 0 and t["entry_form"] == 0
            plan.run()
            assert_same(plan.results(), exp)


@pytest.mark.parametrize("split_min,qpl,persist", [(0, 2, 0), (-1, 2, 0), (-1, 1, 1), (-1, 3, 0), (-700, 2, 1), (-2048, 2, 0),
                                                    (768, 2, 0), (-1, 4, 0), (-700, 4, 0)])
def test_split_pairs_match_oracle(tm, batch, split_min, qpl, persist):
    """Pairs split over two search CTAs (each half of the query groups, winners in global
    memory, the last to finish finalizing): never (0), every pair (-1), most, none in range,
    and the default rule (768: only in batches of fewer pairs than SMs); under each group form
    (a persistent request is set aside when pairs are split); the replay resets the split
    pairs' state."""
    from paper_2511_02036_gb300 import _lib as L
    w, exp = batch
    n_pairs = sum(len(s["nbrs"]) for s in w["steps"])
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        ctx.debug_set(L.TM_DEBUG_SPLIT_MIN, split_min)
        force(tm, ctx, qpl=qpl, persist=persist)
        with ctx.plan(steps_of(w)) as plan:
            t = plan.tuning()
            # a positive threshold splits only in batches of fewer pairs than SMs (152 here)
            active = split_min < 0 or (split_min > 0 and n_pairs < 152)
            n_split = sum(1 for s in w["steps"] for _ in s["nbrs"]
                          if active and w["frames"][s["q"]]["n"] >= abs(split_min))
            assert t["search_units"] == n_pairs + n_split
            for _ in range(3):
                plan.run()
                assert_same(plan.results(), exp)
        assert_same(ctx.batch_run(steps_of(w)), exp)


def test_split_pairs_dense_and_gates(tm):
    """Batches with dense node blocks or the epipole rejection are not split (their instances
    have no split form) and still equal the oracle; without resolve a split batch does."""
    from paper_2511_02036_gb300 import _lib as L
    w = W.make_cfg3b(seed=3520, n_nbrs=4)
    for sp in (tm.SearchParams(dense_min=64), tm.SearchParams(epipole_px=10.0), tm.SearchParams(resolve=False)):
        exp = expected(w, sp)
        with tm.Context(w["cam"], max_kp=2048) as ctx:
            load_all(ctx, w)
            ctx.debug_set(L.TM_DEBUG_SPLIT_MIN, -1)
            with ctx.plan(steps_of(w), sp=sp) as plan:
                plan.run()
                assert_same(plan.results(), exp)


def test_per_lane_form_without_epipolar_gate(tm, batch):
    """The per-lane form's instance without the epipolar gate."""
    w = batch[0]
    sp = tm.SearchParams(epipolar=False)
    exp = expected(w, sp)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        force(tm, ctx, qpl=3)
        with ctx.plan(steps_of(w), sp=sp) as plan:
            assert plan.tuning()["per_lane"] == 1
            plan.run()
            assert_same(plan.results(), exp)
        assert_same(ctx.batch_run(steps_of(w), sp=sp), exp)


@pytest.mark.parametrize("dense_min", [16, 100])
@pytest.mark.parametrize("qpl", [1, 2])
def test_dense_split_matches_oracle(tm, qpl, dense_min):
    """Dense node blocks (tensor cores) beside the candidate rounds under each group width:
    dense_min 16 sends nearly every block to the tensor cores, 100 splits pairs between both."""
    w = W.make_cfg3b(seed=3510, n_nbrs=6)
    sp = tm.SearchParams(dense_min=dense_min)
    exp = expected(w, sp)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        force(tm, ctx, qpl=qpl, persist=1)
        with ctx.plan(steps_of(w), sp=sp) as plan:
            t = plan.tuning()
            assert t["dense_min"] == dense_min and t["dense_split"] >= 1 and t["persistent"] == 0
            plan.run()
            assert_same(plan.results(), exp)


def test_tuned_choice_matches_oracle(tm, batch):
    """The tuner's own choice (measured on this device) and its cached reuse."""
    w, exp = batch
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        with ctx.plan(steps_of(w)) as plan:
            t = plan.tuning()
            assert t["tuned"] == 1 and t["queries_per_warp"] in (32, 64) and t["per_lane"] in (0, 1)
            plan.run()
            assert_same(plan.results(), exp)
        with ctx.plan(steps_of(w)) as plan:
            assert plan.tuning() == t
            plan.run()
            assert_same(plan.results(), exp)


def test_tuning_cache_keyed_by_dense_mode(tm, tmp_path, monkeypatch):
    """A tuning cache file (TM_TUNE_CACHE, first line its key layout) holding other choices for
    batches with dense blocks on than for batches without: in one context a plan with dense
    blocks and then one without each take their own regime's choices (dense blocks fix the
    group form, so their choices must not reach a batch that has every form), and both equal
    the oracle."""
    w = W.make_cfg3b(seed=3510, n_nbrs=6)
    lines = ["tm-tune 2"]
    # key = ((density class x 2 + fewer pairs than SMs) x 3 + dense mode) x 2 + epipole rejection
    for dk in range(-4, 41):
        for few in (0, 1):
            for dmode in range(3):
                for epi in (0, 1):
                    key = ((dk * 2 + few) * 3 + dmode) * 2 + epi
                    # qpl, persistent, prefetch, branch priority, dense_min, dense split divisor
                    kn = (1, 1, 0, 0, 0, 1) if dmode == 1 else (3, 0, 1, 0, 0, 1)
                    lines.append(" ".join(str(v) for v in (key,) + kn))
    path = tmp_path / "tune.txt"
    path.write_text("\n".join(lines) + "\n")
    monkeypatch.setenv("TM_TUNE_CACHE", str(path))
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        for dense_min in (64, 0):
            sp = tm.SearchParams(dense_min=dense_min)
            with ctx.plan(steps_of(w), sp=sp) as plan:
                t = plan.tuning()
                assert t["tuned"] == 1
                if dense_min:
                    assert t["dense_min"] == 64 and t["l2_prefetch"] == 0 and t["per_lane"] == 0
                else:
                    assert t["dense_min"] == 0 and t["l2_prefetch"] == 1 and t["per_lane"] == 1
                plan.run()
                assert_same(plan.results(), expected(w, sp))


@pytest.mark.parametrize("cap,split_min", [(1, 0), (300, 0), (2000, -700), (0, 0)])
@pytest.mark.parametrize("epipolar", [True, False])
def test_entry_form_overflow_matches_oracle(tm, batch, cap, split_min, epipolar):
    """The entry form with an entry list too small for the batch (1 or 300 entries: the pairs
    whose entries did not fit are searched in rounds by their finalize, the others from the
    list; 2000 with split pairs) and sized from the batch (0), with and without the epipolar
    gate: equal to the oracle, replay after replay (the prep kernel resets the count and the
    flags), and the one-shot batch too."""
    from paper_2511_02036_gb300 import _lib as L
    w = batch[0]
    sp = tm.SearchParams(epipolar=epipolar)
    exp = expected(w, sp)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        ctx.debug_set(L.TM_DEBUG_SPLIT_MIN, split_min)
        ctx.debug_set(L.TM_DEBUG_ENTRY_CAP, cap)
        force(tm, ctx, qpl=4)
        with ctx.plan(steps_of(w), sp=sp) as plan:
            assert plan.tuning()["entry_form"] == 1
            for _ in range(3):
                plan.run()
                assert_same(plan.results(), exp)
        assert_same(ctx.batch_run(steps_of(w), sp=sp), exp)
    with pytest.raises(tm.TMError):
        with tm.Context(w["cam"], max_kp=2048) as ctx:
            ctx.debug_set(L.TM_DEBUG_ENTRY_CAP, -1)
