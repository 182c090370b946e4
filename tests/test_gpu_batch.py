"""Batched path (one persistent launch for many steps, CUDA-graph plans, autotuning), the
keyframe store's error behaviour, and full-size cfg2 parity in the benchmark's launch
configuration.  GPU == oracle bit-exactly."""

import ctypes

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


def steps_of(w):
    return [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                 mps=s.get("mps")) for s in w["steps"]]


def oracle_results(w):
    pairs, fuses, cs, cf = [], [], 0, 0
    for st in w["steps"]:
        r, c = O.search_step(w["cam"], w["frames"], st)
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
def small_batch():
    return W.make_cfg2(seed=2100, n_steps=6)


def test_batch_run_small(tm, small_batch):
    w = small_batch
    exp = oracle_results(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        for lanes in (0, 1, 4, 32):
            assert_same(ctx.batch_run(steps_of(w), sp=tm.SearchParams(lanes_per_query=lanes)), exp)
        assert_same(ctx.batch_run(steps_of(w), sp=tm.SearchParams(mode=tm.TM_MODE_PER_PAIR)), exp)


def test_plan_graph_replay(tm, small_batch):
    w = small_batch
    exp = oracle_results(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        with ctx.plan(steps_of(w)) as plan:
            info = plan.info()
            # prep, search (join, evaluation, finalize in the entry form), its copy, fuse, its copy
            assert info["kernels_per_run"] == 5 + 2 * plan.tuning()["entry_form"] and info["ctas"] >= 1
            for _ in range(3):
                plan.run()
                assert_same(plan.results(), exp)
            # a keyframe used by a live plan cannot be removed
            with pytest.raises(tm.TMError) as e:
                ctx.remove_keyframe(w["steps"][0]["q"])
            assert e.value.status == tm.TM_ERR_BUSY
        ctx.remove_keyframe(w["steps"][0]["q"])
        with ctx.plan(steps_of(w)[1:], sp=tm.SearchParams(mode=tm.TM_MODE_PER_PAIR)) as plan:
            plan.run()
            r = plan.results()
            n0 = len(w["steps"][0]["nbrs"])
            for g, e in zip(r.pairs, exp[0][n0:]):
                np.testing.assert_array_equal(g, e)


def test_batch_order_invariance(tm, small_batch):
    """A step's results do not depend on the other steps of the batch nor on their order."""
    w = small_batch
    steps = steps_of(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        full = ctx.batch_run(steps)
        rev = ctx.batch_run(steps[::-1])
        n = [len(s["nbrs"]) for s in steps]
        starts = np.concatenate([[0], np.cumsum(n)])
        rstarts = np.concatenate([[0], np.cumsum(n[::-1])])
        for k in range(len(steps)):
            kk = len(steps) - 1 - k
            for j in range(n[k]):
                np.testing.assert_array_equal(full.pairs[starts[k] + j], rev.pairs[rstarts[kk] + j])
            np.testing.assert_array_equal(full.fuses[k], rev.fuses[kk])
            alone = ctx.batch_run([steps[k]])
            for j in range(n[k]):
                np.testing.assert_array_equal(full.pairs[starts[k] + j], alone.pairs[j])
            np.testing.assert_array_equal(full.fuses[k], alone.fuses[0])


def test_store_errors(tm):
    cam = W.CAM_CFG0
    rng = np.random.default_rng(0)
    a, b = W.random_keyframe(rng, 100, cam), W.random_keyframe(rng, 200, cam)
    with tm.Context(cam, max_kp=256) as ctx:
        ctx.add_keyframe(1, a)
        with pytest.raises(tm.TMError) as e:
            ctx.add_keyframe(1, b)
        assert e.value.status == tm.TM_ERR_EXISTS
        with pytest.raises(tm.TMError) as e:
            ctx.search(1, [9])
        assert e.value.status == tm.TM_ERR_NOT_FOUND
        with pytest.raises(tm.TMError) as e:
            ctx.add_keyframe(2, W.random_keyframe(rng, 300, cam))
        assert e.value.status == tm.TM_ERR_INVALID_ARG
        bad = dict(b)
        bad["level"] = b["level"].copy()
        bad["level"][5] = 9
        with pytest.raises(tm.TMError) as e:
            ctx.add_keyframe(3, bad)
        assert e.value.status == tm.TM_ERR_INVALID_ARG
        ctx.add_keyframe(2, b)
        assert ctx.keyframe_size(2) == 200
        ctx.remove_keyframe(2)
        with pytest.raises(tm.TMError) as e:
            ctx.remove_keyframe(2)
        assert e.value.status == tm.TM_ERR_NOT_FOUND
        # capacity: the C call reports the required count and writes nothing
        a2 = dict(a)
        a2["desc"] = a["desc"].copy()
        ctx.add_keyframe(4, a2)
        nb = np.array([4], np.uint64)
        out = np.full((1, 3), -7, np.int32)
        po = np.zeros(2, np.int32)
        n_out = ctypes.c_size_t()
        sp = tm.SearchParams(ratio_num=0, rot_filter=False, epipolar=False).struct()
        st = tm.tm_search_triangulation(ctx.handle, 1, nb.ctypes.data, 1, ctypes.byref(sp), None, None,
                                        out.ctypes.data, 0, ctypes.byref(n_out), po.ctypes.data, None, None)
        assert st == tm.TM_ERR_CAPACITY and n_out.value == 100 and out[0, 0] == -7


def test_remove_keyframes_all_or_nothing(tm):
    cam = W.CAM_CFG0
    rng = np.random.default_rng(1)
    with tm.Context(cam, max_kp=256) as ctx:
        ctx.add_keyframes([1, 2, 3], [W.random_keyframe(rng, 50 + 10 * k, cam) for k in range(3)])
        for bad, status in (([1, 9], tm.TM_ERR_NOT_FOUND), ([2, 2], tm.TM_ERR_INVALID_ARG)):
            with pytest.raises(tm.TMError) as e:
                ctx.remove_keyframes(bad)
            assert e.value.status == status
        assert [ctx.keyframe_size(i) for i in (1, 2, 3)] == [50, 60, 70]  # nothing removed
        ctx.remove_keyframes([3, 1])
        assert ctx.keyframe_size(2) == 60
        for i in (1, 3):
            with pytest.raises(tm.TMError):
                ctx.keyframe_size(i)
        ctx.remove_keyframes([])


def test_step_table_batches(tm, small_batch):
    """A batch described by a StepTable (columns) gives the same results as step dicts."""
    w = small_batch
    exp = oracle_results(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        st_arr, masks, mps, _keep = tm.pack_batch(steps_of(w), ctx.sizes)
        table = tm.StepTable(np.array([st_arr[k].kf_id for k in range(len(w["steps"]))], np.uint64),
                             np.array([len(s["nbrs"]) for s in w["steps"]], np.int32),
                             np.concatenate([np.asarray(s["nbrs"], np.uint64) for s in w["steps"]]),
                             np.array([st_arr[k].q_free_off for k in range(len(w["steps"]))]),
                             np.array([st_arr[k].nbr_free_off for k in range(len(w["steps"]))]),
                             np.array([st_arr[k].mp_begin for k in range(len(w["steps"]))], np.int32),
                             np.array([st_arr[k].mp_count for k in range(len(w["steps"]))], np.int32))
        assert_same(ctx.batch_run(table, masks=masks, mps=mps), exp)
        with ctx.plan(table, masks=masks, mps=mps) as plan:
            plan.run()
            assert_same(plan.results(), exp)


def test_memory_budget_admission(tm):
    cam = W.CAM_CFG0
    rng = np.random.default_rng(1)
    with tm.Context(cam, max_kp=512) as probe:
        slot = probe.stats()["slot_bytes"]
    with tm.Context(cam, max_kp=512, budget=3 * slot + 10) as ctx:
        for k in range(3):
            ctx.add_keyframe(k, W.random_keyframe(rng, 300, cam))
        with pytest.raises(tm.TMError) as e:
            ctx.add_keyframe(3, W.random_keyframe(rng, 300, cam))
        assert e.value.status == tm.TM_ERR_NO_MEMORY
        # all-or-nothing batched add
        with pytest.raises(tm.TMError):
            ctx.add_keyframes([7, 8], [W.random_keyframe(rng, 10, cam)] * 2)
        assert ctx.stats()["slots_used"] == 3
        ctx.remove_keyframe(0)
        ctx.add_keyframe(3, W.random_keyframe(rng, 300, cam))
        assert ctx.stats()["slots_used"] == 3


def test_store_reserve(tm):
    """tm_store_reserve allocates slots ahead within the budget (one allocation); later
    additions take them without growing the store; beyond the budget it reports NO_MEMORY and
    keeps what fits."""
    cam = W.CAM_CFG0
    rng = np.random.default_rng(2)
    with tm.Context(cam, max_kp=512) as probe:
        slot = probe.stats()["slot_bytes"]
    with tm.Context(cam, max_kp=512, budget=10 * slot) as ctx:
        ctx.reserve(8)
        st = ctx.stats()
        assert st["bytes_reserved"] == 8 * slot and st["slots_used"] == 0
        ctx.reserve(4)  # already free: nothing allocated
        assert ctx.stats()["bytes_reserved"] == 8 * slot
        for k in range(8):
            ctx.add_keyframe(k, W.random_keyframe(rng, 100, cam))
        assert ctx.stats()["bytes_reserved"] == 8 * slot
        with pytest.raises(tm.TMError) as e:
            ctx.reserve(5)
        assert e.value.status == tm.TM_ERR_NO_MEMORY
        assert ctx.stats()["bytes_reserved"] == 10 * slot
        for k in range(8, 10):
            ctx.add_keyframe(k, W.random_keyframe(rng, 100, cam))
        with pytest.raises(tm.TMError) as e:
            ctx.add_keyframe(10, W.random_keyframe(rng, 100, cam))
        assert e.value.status == tm.TM_ERR_NO_MEMORY


@pytest.fixture(scope="module")
def cfg2():
    return W.make_cfg2()


def test_cfg2_full_size_parity(tm, cfg2):
    """The benchmark's workload (64 steps, 821 pairs, 537k map points) in the benchmark's
    launch configuration (autotuned plan, CUDA graph): every pair and every step equals the
    oracle."""
    w = cfg2
    exp = oracle_results(w)
    new_ids = [s["q"] for s in w["steps"]]
    old_ids = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        ctx.add_keyframes(old_ids, [w["frames"][i] for i in old_ids])
        with ctx.plan(steps_of(w), new=(new_ids, [w["frames"][i] for i in new_ids])) as plan:
            plan.run()
            plan.run()
            assert_same(plan.results(), exp)
            assert all(t == 0 for t in plan.stage_times())  # untimed graph: no events
            plan.run(timed=True)
            assert_same(plan.results(), exp)
            ms = plan.stage_times()
            assert len(ms) == 6 and all(t > 0 for t in ms[:4]) and ms[4] == 0 and ms[5] > 0  # no dense blocks


def test_new_keyframes_enter_with_the_batch(tm, small_batch):
    """The steps' new keyframes are ingested in the batch's own launch sequence (one-shot and
    replayed by a plan's graph): same results; on failure they are not stored."""
    w = small_batch
    exp = oracle_results(w)
    new_ids = [s["q"] for s in w["steps"]]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        old = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        new = (new_ids, [w["frames"][i] for i in new_ids])
        assert_same(ctx.batch_run(steps_of(w), new=new), exp)
        assert ctx.keyframe_size(new_ids[0]) == w["frames"][new_ids[0]]["n"]
        # already stored now: the call fails and stores nothing more
        with pytest.raises(tm.TMError) as e:
            ctx.batch_run(steps_of(w), new=new)
        assert e.value.status == tm.TM_ERR_EXISTS
        for i in new_ids:
            ctx.remove_keyframe(i)
        # a failing batch (unknown neighbour) leaves the new keyframes out of the store
        bad = steps_of(w)
        bad[0] = dict(bad[0], nbrs=[10 ** 9])
        with pytest.raises(tm.TMError):
            ctx.batch_run(bad, new=new)
        with pytest.raises(tm.TMError):
            ctx.keyframe_size(new_ids[0])
        with ctx.plan(steps_of(w), new=new) as plan:
            # ingest, prep, search (three launches in the entry form), its copy, fuse, its copy
            assert plan.info()["kernels_per_run"] == 6 + 2 * plan.tuning()["entry_form"]
            for _ in range(3):
                plan.run()
                assert_same(plan.results(), exp)


def test_bounded_wait_reports_timeout(tm, small_batch):
    """Failure detection without a GPU fault: the search and fusion kernels' bounded waits are
    made to run out (a barrier that nothing arrives at, after the copies have landed); the
    call reports TM_ERR_TIMEOUT, stores nothing, and the context keeps working."""
    from paper_2511_02036_gb300 import _lib as L
    w = small_batch
    exp = oracle_results(w)
    new_ids = [s["q"] for s in w["steps"]]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        old = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        ctx.debug_set(L.TM_DEBUG_WAIT_LIMIT, 20_000_000)  # ~10 ms of SM clock
        ctx.debug_set(L.TM_DEBUG_STARVE_WAITS, 1)
        with pytest.raises(tm.TMError) as e:
            ctx.batch_run(steps_of(w), new=(new_ids, [w["frames"][i] for i in new_ids]))
        assert e.value.status == tm.TM_ERR_TIMEOUT
        with pytest.raises(tm.TMError):
            ctx.keyframe_size(new_ids[0])  # the failed batch stored nothing
        ctx.debug_set(L.TM_DEBUG_STARVE_WAITS, 0)
        assert_same(ctx.batch_run(steps_of(w), new=(new_ids, [w["frames"][i] for i in new_ids])), exp)
        with pytest.raises(tm.TMError) as e:
            ctx.debug_set(99, 1)
        assert e.value.status == tm.TM_ERR_INVALID_ARG


def test_pinned_host_inputs(tm, small_batch):
    """New keyframes, masks and map points in page-locked host memory (torch pinned tensors):
    the keyframes are gathered by a kernel straight from host memory; results equal the
    oracle's, twice in a row (the context's reused result buffers)."""
    torch = pytest.importorskip("torch")
    w = small_batch
    exp = oracle_results(w)
    new_ids = [s["q"] for s in w["steps"]]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        old = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        st_arr, masks, mps, _keep = tm.pack_batch(steps_of(w), ctx.sizes)
        steps = [dict(kf_id=st_arr[k].kf_id, nbrs=w["steps"][k]["nbrs"], q_free_off=st_arr[k].q_free_off,
                      nbr_free_off=st_arr[k].nbr_free_off, mp_begin=st_arr[k].mp_begin,
                      mp_count=st_arr[k].mp_count) for k in range(len(w["steps"]))]
        h_mps = {k: (pin(v) if isinstance(v, np.ndarray) else v) for k, v in mps.items()}
        h_new = [dict(desc=pin(f["desc"]), xy=pin(f["xy"]), angle=pin(f["angle"]), level=pin(f["level"]),
                      node=pin(f["node"].view(np.int32)), Tcw=f["Tcw"]) for f in (w["frames"][i] for i in new_ids)]
        fr = [w["frames"][i] for i in new_ids]
        packed = dict(n=[f["n"] for f in fr], desc=pin(np.concatenate([f["desc"] for f in fr])),
                      xy=pin(np.concatenate([f["xy"] for f in fr])), angle=pin(np.concatenate([f["angle"] for f in fr])),
                      level=pin(np.concatenate([f["level"] for f in fr])),
                      node=pin(np.concatenate([f["node"] for f in fr]).view(np.int32)),
                      Tcw=np.stack([np.asarray(f["Tcw"], np.float64).reshape(12) for f in fr]))
        for new in (h_new, h_new, packed):
            assert_same(ctx.batch_run(steps, masks=pin(masks), mps=h_mps, new=(new_ids, new)), exp)
            for i in new_ids:
                ctx.remove_keyframe(i)


@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
def test_packed_new_keyframes(tm, small_batch, kind):
    """The new keyframes as one packed record (tm_keyframes_packed) in pageable host,
    page-locked host and device memory: one-shot batches and a plan give the oracle's results;
    a packed set whose arrays sit in different kinds of memory, a level above 7 and a count
    above the capacity are refused before any work, and the store is left as it was."""
    torch = pytest.importorskip("torch")
    w = small_batch
    exp = oracle_results(w)
    new_ids = [s["q"] for s in w["steps"]]
    fr = [w["frames"][i] for i in new_ids]
    cat = lambda k: np.ascontiguousarray(np.concatenate([f[k] for f in fr]))  # noqa: E731
    host = dict(desc=cat("desc"), xy=cat("xy"), angle=cat("angle"), level=cat("level"), node=cat("node"))
    put = {"pageable": lambda a: a, "pinned": lambda a: torch.from_numpy(a).pin_memory(),
           "device": lambda a: torch.from_numpy(a).cuda()}[kind]
    packed = {k: put(v) for k, v in host.items()}
    packed["n"] = [f["n"] for f in fr]
    packed["Tcw"] = np.stack([np.asarray(f["Tcw"], np.float64).reshape(12) for f in fr])
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        old = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        used = ctx.stats()["slots_used"]
        for _ in range(2):
            assert_same(ctx.batch_run(steps_of(w), new=(new_ids, packed)), exp)
            ctx.remove_keyframes(new_ids)
        with ctx.plan(steps_of(w), new=(new_ids, packed)) as plan:
            plan.run()
            assert_same(plan.results(), exp)
        ctx.remove_keyframes(new_ids)
        bad = []
        mixed = dict(packed)
        mixed["level"] = torch.from_numpy(host["level"]).cuda() if kind != "device" else host["level"]
        bad.append(mixed)
        if kind != "device":
            lv = dict(packed)
            lv_arr = host["level"].copy()
            lv_arr[len(lv_arr) // 2] = 8
            lv["level"] = put(lv_arr)
            bad.append(lv)
        big = dict(packed)
        big["n"] = list(packed["n"])
        big["n"][0] = 4096
        bad.append(big)
        for b in bad:
            with pytest.raises(tm.TMError) as e:
                ctx.batch_run(steps_of(w), new=(new_ids, b))
            assert e.value.status == tm.TM_ERR_INVALID_ARG
            assert ctx.stats()["slots_used"] == used
        assert_same(ctx.batch_run(steps_of(w), new=(new_ids, packed)), exp)


def test_async_batches(tm, small_batch):
    """tm_batch_begin / tm_batch_finish: batches in flight at once, the second using as
    neighbour a keyframe that the first stores; finished out of order, each equal to the
    oracle.  A begin beyond TM_BATCH_INFLIGHT is refused, the keyframes in-flight batches use
    cannot be removed, an unknown ticket is refused, and a pipelined loop (begin k + 1, then
    finish k) gives the oracle's results at every step, also as views into two caller-owned
    result buffer sets taken in turn (out=)."""
    from paper_2511_02036_gb300 import _lib as L
    w = small_batch
    st = w["steps"]
    nb1 = st[1]["nbrs"][0]  # stored by the first batch, read by the second
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        old = sorted(set(i for s in st for i in s["nbrs"]) - {nb1})
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        s0, s1 = steps_of(dict(w, steps=st[:1])), steps_of(dict(w, steps=st[1:2]))
        t0 = ctx.batch_begin(s0, new=([st[0]["q"], nb1], [w["frames"][st[0]["q"]], w["frames"][nb1]]))
        t1 = ctx.batch_begin(s1, new=([st[1]["q"]], [w["frames"][st[1]["q"]]]))
        # fill the remaining slots with searches of already stored keyframes, then one more
        extra = [ctx.batch_begin(steps_of(dict(w, steps=st[1:2])), sp=tm.SearchParams())
                 for _ in range(L.TM_BATCH_INFLIGHT - 2)]
        with pytest.raises(tm.TMError) as e:
            ctx.batch_begin(steps_of(dict(w, steps=st[2:3])))
        assert e.value.status == tm.TM_ERR_BUSY
        exp1 = oracle_results(dict(w, steps=st[1:2]))
        for t in extra:
            assert_same(ctx.batch_finish(t), exp1)
        with pytest.raises(tm.TMError) as e:
            ctx.remove_keyframe(st[1]["nbrs"][1])
        assert e.value.status == tm.TM_ERR_BUSY
        # keyframes that batches in flight are still storing: only later asynchronous batches
        # (ordered after their ingest) may read them; other calls are refused until finished
        with pytest.raises(tm.TMError) as e:
            ctx.batch_run(s1)
        assert e.value.status == tm.TM_ERR_BUSY
        with pytest.raises(tm.TMError) as e:
            ctx.search(st[1]["q"], st[1]["nbrs"])
        assert e.value.status == tm.TM_ERR_BUSY
        r1 = ctx.batch_finish(t1)
        r0 = ctx.batch_finish(t0)
        for res, part in ((r0, st[:1]), (r1, st[1:2])):
            assert_same(res, oracle_results(dict(w, steps=part)))
        r = L.tm_batch_result()
        assert tm.tm_batch_finish(ctx.handle, t0, ctypes.byref(r)) == tm.TM_ERR_NOT_FOUND  # finished already
        # pipelined: begin step k + 1 before finishing step k (all remaining steps, two id sets)
        ctx.remove_keyframes([st[0]["q"], st[1]["q"]])
        rest = st[2:]
        prev = None
        got = []
        for k, s in enumerate(rest):
            t = ctx.batch_begin(steps_of(dict(w, steps=[s])), new=([s["q"]], [w["frames"][s["q"]]]))
            if prev is not None:
                got.append(ctx.batch_finish(prev))
            prev = t
        got.append(ctx.batch_finish(prev))
        for res, s in zip(got, rest):
            assert_same(res, oracle_results(dict(w, steps=[s])))
        # the same loop with the results as views into caller-owned buffers, checked as each
        # arrives (the set is written again two batches later)
        ctx.remove_keyframes([s["q"] for s in rest])
        outs = [tm.ResultBuffers(), tm.ResultBuffers()]
        prev = None

        def take(t, k):
            res = ctx.batch_finish(t, out=outs[k % 2])
            for a, b in ((res.matches, outs[k % 2].m), (res.fuse, outs[k % 2].f)):
                assert len(a) == 0 or np.shares_memory(a, b)
            assert_same(res, oracle_results(dict(w, steps=[rest[k]])))

        for k, s in enumerate(rest):
            t = ctx.batch_begin(steps_of(dict(w, steps=[s])), new=([s["q"]], [w["frames"][s["q"]]]))
            if prev is not None:
                take(prev, k - 1)
            prev = t
        take(prev, len(rest) - 1)
        ctx.remove_keyframes([s["q"] for s in rest])
        res = ctx.batch_run(steps_of(dict(w, steps=rest[:1])), new=([rest[0]["q"]], [w["frames"][rest[0]["q"]]]),
                            out=outs[0])
        assert len(res.matches) == 0 or np.shares_memory(res.matches, outs[0].m)
        assert_same(res, oracle_results(dict(w, steps=rest[:1])))
        assert L.TM_BATCH_INFLIGHT == 4


def test_async_batches_two_threads(tm, small_batch):
    """A producer thread begins batches (at most three in flight) while a consumer thread
    finishes them in order, into its own result buffers, and removes their keyframes: every
    batch equals the oracle (tm_batch_finish waits without holding the context)."""
    import queue
    import threading
    w = small_batch
    st = w["steps"]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        old = sorted(set(i for s in st for i in s["nbrs"]))
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        exp = [oracle_results(dict(w, steps=[s])) for s in st]
        # each batch stores its step's new keyframe under an id of its own round, not one of the
        # stored ids
        rounds, depth = 4, 3
        outs = [tm.ResultBuffers() for _ in range(depth)]
        sem, q, got, err = threading.Semaphore(depth), queue.Queue(), [], []

        def consumer():
            while True:
                item = q.get()
                if item is None:
                    return
                t, k, nid = item
                try:
                    res = ctx.batch_finish(t, out=outs[k % depth])
                    got.append((k, [a.copy() for a in res.pairs], [a.copy() for a in res.fuses],
                                res.n_comparisons_search, res.n_comparisons_fuse))
                    ctx.remove_keyframes([nid])
                except BaseException as ex:  # noqa: BLE001
                    err.append(ex)
                sem.release()

        th = threading.Thread(target=consumer)
        th.start()
        try:
            n = 0
            for r in range(rounds):
                for s in st:
                    sem.acquire()
                    nid = s["q"] + ((r + 1) << 40)
                    step = dict(kf_id=nid, nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                                mps=s.get("mps"))
                    q.put((ctx.batch_begin([step], new=([nid], [w["frames"][s["q"]]])), n, nid))
                    n += 1
        finally:
            q.put(None)
            th.join()
        assert not err, err
        assert [k for k, *_ in got] == list(range(rounds * len(st)))
        for k, pairs, fuses, cs, cf in got:
            e_pairs, e_fuses, e_cs, e_cf = exp[k % len(st)]
            assert len(pairs) == len(e_pairs) and len(fuses) == len(e_fuses)
            for g, e in zip(pairs, e_pairs):
                np.testing.assert_array_equal(g, e)
            for g, e in zip(fuses, e_fuses):
                np.testing.assert_array_equal(g, e)
            assert cs == e_cs and cf == e_cf


def forward_steps(w, skip=True):
    return [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                 mps=s.get("mps"), fwd_mps=s["fwd_mps"], fwd_skip=s["fwd_skip"] if skip else None)
            for s in w["steps"]]


def oracle_forward(w, skip=True):
    out, ncmp = [], 0
    for st in w["steps"]:
        s2 = dict(st)
        if not skip:
            s2["fwd_skip"] = None
        r, c = O.fuse_forward_step(w["cam"], w["frames"], s2)
        out.extend(r)
        ncmp += c
    return out, ncmp


@pytest.mark.parametrize("mode", [0, 1])
def test_forward_fusion_batch(tm, mode):
    """Forward fusion (the new keyframes' map points into every neighbour, with per-neighbour
    skip bytes) beside the search and the backward fusion: every array equals the oracle's."""
    w = W.make_cfg2(seed=2200, n_steps=5, forward=True)
    exp = oracle_results(w)
    efw, ecw = oracle_forward(w)
    assert sum(len(x) for x in efw) > 100
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        res = ctx.batch_run(forward_steps(w), sp=tm.SearchParams(mode=mode))
        assert_same(res, exp)
        assert len(res.fwds) == len(efw)
        for g, e in zip(res.fwds, efw):
            np.testing.assert_array_equal(g, e)
        assert res.n_comparisons_fwd == ecw
        # no skip bytes: every map point into every neighbour
        efw2, ecw2 = oracle_forward(w, skip=False)
        res2 = ctx.batch_run(forward_steps(w, skip=False), sp=tm.SearchParams(mode=mode))
        for g, e in zip(res2.fwds, efw2):
            np.testing.assert_array_equal(g, e)
        assert res2.n_comparisons_fwd == ecw2 and ecw2 > ecw


def test_forward_fusion_plan_and_mixed_steps(tm):
    """A plan with forward fusion, and a batch where only some steps ask for it (their pairs
    get empty forward lists)."""
    w = W.make_cfg2(seed=2201, n_steps=4, forward=True)
    exp = oracle_results(w)
    efw, ecw = oracle_forward(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        with ctx.plan(forward_steps(w)) as plan:
            for _ in range(2):
                plan.run()
                r = plan.results()
                assert_same(r, exp)
                for g, e in zip(r.fwds, efw):
                    np.testing.assert_array_equal(g, e)
                assert r.n_comparisons_fwd == ecw
        steps = forward_steps(w)
        for k in (1, 3):
            steps[k] = {key: v for key, v in steps[k].items() if key not in ("fwd_mps", "fwd_skip")}
        r = ctx.batch_run(steps)
        p = 0
        for k, st in enumerate(w["steps"]):
            for j in range(len(st["nbrs"])):
                e = efw[p] if k not in (1, 3) else np.zeros((0, 3), np.int32)
                np.testing.assert_array_equal(r.fwds[p], e)
                p += 1


def test_fuse_apply_consumes_batch_lists(tm):
    """The GPU's fusion lists feed the sequential fuse-apply (Sec. IV-D) in ORB-SLAM's order: the
    new keyframe's map points into each neighbour in turn, then the neighbours' map points into
    the new keyframe.  The library's host map after the GPU lists equals the oracle's map after
    the oracle's lists.  The map's starting observations are drawn at random (a valid state)."""
    w = W.make_cfg2(seed=2202, n_steps=1, forward=True)
    st = w["steps"][0]
    efw, _ = oracle_forward(w)
    efu = oracle_results(w)[1][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        res = ctx.batch_run(forward_steps(w))
    q, nbrs = st["q"], list(st["nbrs"])
    nf, nb = int(st["fwd_mps"]["n"]), int(st["mps"]["n"])
    fwd_ids = np.arange(nf, dtype=np.int32)
    bwd_ids = np.arange(nf, nf + nb, dtype=np.int32)
    rng = np.random.default_rng(2202)
    fm = O.FuseMap()
    for k in [q] + nbrs:
        fm.add_keyframe(k, w["frames"][k]["n"], w["frames"][k]["level"])
    triples = []

    def observe(k, m):
        free = [j for j, x in enumerate(fm.kp[k]) if x is None]
        if free and k not in fm.obs.get(m, {}):
            j = int(rng.choice(free))
            fm.observe(k, j, m)
            triples.append((k, j, m))
    for i in range(nf):
        observe(q, int(fwd_ids[i]))
        for n, k in enumerate(nbrs):
            if st["fwd_skip"][n][i]:
                observe(k, int(fwd_ids[i]))
    for i in range(nb):
        for k in rng.choice(nbrs, size=int(rng.integers(1, 3)), replace=False):
            observe(int(k), int(bwd_ids[i]))
        for k in rng.permutation(nbrs):  # every candidate's point must exist
            if int(bwd_ids[i]) not in fm.obs:
                observe(int(k), int(bwd_ids[i]))
    assert all(m in fm.obs for m in range(nf + nb))
    with tm.Map(nf + nb) as mp:
        for k in [q] + nbrs:
            mp.add_keyframe(k, w["frames"][k]["n"], w["frames"][k]["level"])
            t = [(j, m) for (kk, j, m) in triples if kk == k]
            mp.add_observations(k, [j for j, _ in t], [m for _, m in t])
        totals = {}
        for n, k in enumerate(nbrs):
            est = fm.fuse(k, [(int(fwd_ids[a]), int(j)) for a, j, _ in efw[n]])
            assert mp.fuse_apply(k, res.fwds[n], fwd_ids) == est
            for f, v in est.items():
                totals[f] = totals.get(f, 0) + v
        est = fm.fuse(q, [(int(bwd_ids[a]), int(j)) for a, j, _ in efu])
        assert mp.fuse_apply(q, res.fuses[0], bwd_ids) == est
        assert totals["added"] > 0 and est["added"] + est["replaced_existing"] + est["merged_into_existing"] > 0
        for k in [q] + nbrs:
            np.testing.assert_array_equal(mp.keyframe_points(k, w["frames"][k]["n"]),
                                          [-1 if x is None else x for x in fm.kp[k]])
        live, cur, nobs = mp.point_info(np.arange(nf + nb))
        for m in range(nf + nb):
            c = fm.current(m)
            assert cur[m] == (-1 if c is None else c) and nobs[m] == len(fm.obs.get(m, {}))


def check_points(w, res, exp_pairs, params=None):
    p = 0
    for st in w["steps"]:
        for f in st["nbrs"]:
            xyz, ok = O.triangulate(w["cam"], w["frames"][st["q"]], w["frames"][f], exp_pairs[p], params)
            a, b = res.pair_offsets[p], res.pair_offsets[p + 1]
            np.testing.assert_array_equal(res.points[a:b], xyz)
            np.testing.assert_array_equal(res.point_ok[a:b], ok)
            p += 1


@pytest.mark.parametrize("mode", [0, 1])
def test_triangulation_batch(tm, small_batch, mode):
    """Triangulation and acceptance of every match on the GPU (float32, fixed order) equals the
    oracle's bit for bit: points (float32) and accepted flags, batched and per-pair forms."""
    w = small_batch
    exp = oracle_results(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        res = ctx.batch_run(steps_of(w), sp=tm.SearchParams(mode=mode), tri=tm.TriParams())
        assert_same(res, exp)
        assert res.point_ok.sum() > 100
        check_points(w, res, exp[0])
        tight = tm.TriParams(cos_parallax_max=0.999, chi2=2.0)
        res2 = ctx.batch_run(steps_of(w), sp=tm.SearchParams(mode=mode), tri=tight)
        check_points(w, res2, exp[0], O.TriParams(0.999, 2.0))
        assert res2.point_ok.sum() < res.point_ok.sum()


def test_triangulation_plan_new_keyframes(tm, small_batch):
    """In a plan whose new keyframes enter the store with the batch (their slots are written by
    the batch's own ingest before the triangulation reads them)."""
    w = small_batch
    exp = oracle_results(w)
    new_ids = [s["q"] for s in w["steps"]]
    old_ids = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        ctx.add_keyframes(old_ids, [w["frames"][i] for i in old_ids])
        with ctx.plan(steps_of(w), new=(new_ids, [w["frames"][i] for i in new_ids]), tri=tm.TriParams()) as plan:
            # ingest, prep, search (three launches in the entry form), its copy, triangulation, fuse,
            # its copy
            assert plan.info()["kernels_per_run"] == 7 + 2 * plan.tuning()["entry_form"]
            for _ in range(2):
                plan.run()
                r = plan.results()
                assert_same(r, exp)
                check_points(w, r, exp[0])


@pytest.mark.parametrize("mode", [0, 1])
def test_pair_baseline_skip_batch(tm, small_batch, mode):
    """ORB-family pair-baseline skip: per neighbour a median scene depth chosen so that every
    other pair falls below the ratio; skipped pairs are empty and cost no comparisons, the
    others equal the oracle's."""
    w = small_batch
    steps = []
    ow = dict(w)
    ow["steps"] = []
    for s in w["steps"]:
        cq = W.camera_center(w["frames"][s["q"]]["Tcw"])
        md = []
        for k, f in enumerate(s["nbrs"]):
            base = float(np.linalg.norm(cq - W.camera_center(w["frames"][f]["Tcw"])))
            md.append(base / 0.01 * (1.5 if k % 2 == 0 else 0.5))
        s2 = dict(s)
        s2["nbr_median_depth"] = np.array(md, np.float32)
        ow["steps"].append(s2)
        steps.append(dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                          mps=s.get("mps"), nbr_median_depth=s2["nbr_median_depth"]))
    sp = tm.SearchParams(baseline_min_ratio=0.01, mode=mode)
    osp = O.SearchParams(baseline_min_ratio=0.01)
    exp, ecmp = [], 0
    for st in ow["steps"]:
        r, c = O.search_step(w["cam"], w["frames"], st, osp)
        exp.extend(r)
        ecmp += c
    assert sum(len(e) == 0 for e in exp) >= len(exp) // 2 - 1
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        res = ctx.batch_run(steps, sp=sp)
        for g, e in zip(res.pairs, exp):
            np.testing.assert_array_equal(g, e)
        assert res.n_comparisons_search == ecmp


@pytest.mark.parametrize("kind", ["pinned", "device"])
def test_mappoint_block(tm, small_batch, kind):
    """The batch's map points in one staging block (pack_mappoints; tm_batch_inputs.mps_block:
    one upload), page-locked host or device memory: one-shot, asynchronous and plan batches give
    the oracle's results; a descriptor array off its 16-byte alignment in the block and an array
    outside the block are refused before any work."""
    torch = pytest.importorskip("torch")
    w = small_batch
    exp = oracle_results(w)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_all(ctx, w)
        st_arr, masks, mps, _keep = tm.pack_batch(steps_of(w), ctx.sizes)
        steps = [dict(kf_id=st_arr[k].kf_id, nbrs=w["steps"][k]["nbrs"], q_free_off=st_arr[k].q_free_off,
                      nbr_free_off=st_arr[k].nbr_free_off, mp_begin=st_arr[k].mp_begin,
                      mp_count=st_arr[k].mp_count) for k in range(len(w["steps"]))]
        fields = ("pos", "normal", "desc", "min_dist", "max_dist", "skip")
        blk = tm.pack_mappoints(mps, pinned=True)
        if kind == "device":
            # the same layout in device memory: views at the host block's offsets
            dev_block = blk["block"].cuda()
            dv = {}
            for f in fields:
                if f in blk:
                    off = blk[f].data_ptr() - blk["block"].data_ptr()
                    nb = blk[f].numel() * blk[f].element_size()
                    dv[f] = dev_block[off:off + nb].view(blk[f].dtype).view(blk[f].shape)
            blk = dict(n=blk["n"], block=dev_block, **dv)
        d_masks = torch.from_numpy(np.ascontiguousarray(masks)).cuda()
        assert_same(ctx.batch_run(steps, masks=d_masks, mps=blk), exp)
        t = ctx.batch_begin(steps, masks=d_masks, mps=blk)
        assert_same(ctx.batch_finish(t), exp)
        with ctx.plan(steps, masks=d_masks, mps=blk) as plan:
            plan.run()
            assert_same(plan.results(), exp)
        if kind == "pinned":
            # desc 8 bytes into its slot: off the 16-byte alignment
            n = int(mps["n"])
            raw = blk["block"]
            shifted = torch.empty(raw.numel() + 64, dtype=torch.uint8).pin_memory()
            shifted[:raw.numel()] = raw
            bad = dict(n=n, block=shifted)
            for f in fields:
                if f in blk:
                    o = blk[f].data_ptr() - raw.data_ptr() + (8 if f == "desc" else 0)
                    nb = blk[f].numel() * blk[f].element_size()
                    bad[f] = shifted[o:o + nb].view(blk[f].dtype).view(blk[f].shape)
            with pytest.raises(tm.TMError) as e:
                ctx.batch_run(steps, masks=d_masks, mps=bad)
            assert e.value.status == tm.TM_ERR_INVALID_ARG
            # an array outside the block
            outside = dict(blk, desc=torch.from_numpy(np.ascontiguousarray(mps["desc"])).pin_memory())
            with pytest.raises(tm.TMError) as e:
                ctx.batch_run(steps, masks=d_masks, mps=outside)
            assert e.value.status == tm.TM_ERR_INVALID_ARG
            assert_same(ctx.batch_run(steps, masks=d_masks, mps=blk), exp)
