"""Continuous-batching server: requests admitted while others run on the GPU give the same
results as the oracle (= each request alone), admission by store memory with eviction, and
errors reported per request."""

import time

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


@pytest.fixture(scope="module")
def stream():
    return W.make_stream_cfg4(seed=4100, n_kf=60, duration_s=12.0)


def submit_all(srv, w, rate_hz=None, rng=None):
    tickets = []
    t0 = time.perf_counter()
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, len(w["steps"]))) if rate_hz else None
    for k, st in enumerate(w["steps"]):
        if arrivals is not None:
            while time.perf_counter() - t0 < arrivals[k]:
                time.sleep(2e-4)
        f = w["frames"][st["q"]]
        tickets.append(srv.submit(st["q"], f, st["nbrs"], st["q_free"], st["nbr_free"], st["mps"]))
    return tickets


def check_against_oracle(srv, w, tickets):
    lat = []
    for st, t in zip(w["steps"], tickets):
        pairs, fuse, info = srv.take(t)
        assert info["status"] == 0
        exp, _ = O.search_step(w["cam"], w["frames"], st)
        assert len(pairs) == len(exp)
        for g, e in zip(pairs, exp):
            np.testing.assert_array_equal(g, e)
        fe, _ = O.fuse_step(w["cam"], w["frames"], st)
        np.testing.assert_array_equal(fuse, fe)
        lat.append(info["t_done"] - info["t_submit"])
    return np.array(lat)


@pytest.mark.parametrize("batch,inflight,rate", [(64, 3, None), (4, 2, 400.0), (1, 1, None)])
def test_stream_matches_oracle(tm, stream, batch, inflight, rate):
    w = stream
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        with ctx.server(max_batch_requests=batch, max_inflight_batches=inflight) as srv:
            tickets = submit_all(srv, w, rate, np.random.default_rng(0))
            lat = check_against_oracle(srv, w, tickets)
    assert np.all(lat > 0)


@pytest.mark.parametrize("batch", [2, 8])
def test_admission_by_memory_with_eviction(tm, stream, batch):
    """A store that holds only 24 keyframes: the server evicts the oldest (neighbours reach
    back at most 20) and every request still completes correctly.  The counters show the
    store bounded by its budget while all 60 keyframes pass through it (whether a request
    also had to wait for a slot depends on how fast requests arrive against the GPU, so the
    deferral count is only reported)."""
    w = stream
    with tm.Context(w["cam"], max_kp=2048) as probe:
        slot = probe.stats()["slot_bytes"]
    with tm.Context(w["cam"], max_kp=2048, budget=24 * slot) as ctx:
        with ctx.server(max_batch_requests=batch, max_inflight_batches=2, evict_after=21) as srv:
            tickets = submit_all(srv, w)
            check_against_oracle(srv, w, tickets)
            s = srv.stats()
        assert ctx.stats()["slots_used"] <= 24
    n = len(w["steps"])
    assert s["submitted"] == s["admitted"] == s["completed"] == n and s["failed"] == 0
    assert s["store_slot_limit"] == 24 and 21 <= s["peak_store_slots"] <= 24
    assert s["evicted"] >= n - 24 and 1 <= s["peak_inflight"] <= 2
    assert n / batch <= s["batches"] <= n and s["deferrals"] >= 0


def test_request_errors(tm, stream):
    w = stream
    st = w["steps"][5]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        with ctx.server() as srv:
            # neighbours never stored -> NOT_FOUND for this request only
            t = srv.submit(st["q"], w["frames"][st["q"]], st["nbrs"])
            info = srv.poll(t, timeout=60.0)
            assert info["done"] and info["status"] == tm.TM_ERR_NOT_FOUND
            with pytest.raises(tm.TMError):
                srv.take(t)
            # the first keyframe has no neighbours and succeeds
            s0 = w["steps"][0]
            t0 = srv.submit(s0["q"], w["frames"][s0["q"]], [], mps=None)
            pairs, fuse, info = srv.take(t0)
            assert info["status"] == 0 and pairs == [] and len(fuse) == 0
            # the same keyframe id again -> EXISTS
            t1 = srv.submit(s0["q"], w["frames"][s0["q"]], [])
            assert srv.poll(t1, timeout=60.0)["status"] == tm.TM_ERR_EXISTS
            # neighbour masks shorter than the neighbours' keypoints -> INVALID_ARG for that
            # request alone; the next request (same neighbours, full masks) is served
            s1 = w["steps"][1]
            short = np.concatenate([np.asarray(m, np.uint8) for m in s1["nbr_free"]])[:-1]
            t2 = srv.submit(s1["q"], w["frames"][s1["q"]], s1["nbrs"], s1["q_free"], short, s1["mps"])
            assert srv.poll(t2, timeout=60.0)["status"] == tm.TM_ERR_INVALID_ARG
            t3 = srv.submit(s1["q"], w["frames"][s1["q"]], s1["nbrs"], s1["q_free"], s1["nbr_free"], s1["mps"])
            pairs, fuse, info = srv.take(t3)
            assert info["status"] == 0
            exp, _ = O.search_step(w["cam"], w["frames"], s1)
            for g, e in zip(pairs, exp):
                np.testing.assert_array_equal(g, e)


@pytest.mark.parametrize("batch,skip", [(8, True), (1, False)])
def test_forward_fusion_and_triangulation_served(tm, batch, skip):
    """Requests carrying their new keyframe's own map points (forward fusion into every
    neighbour, with or without per-neighbour skip bytes), served with triangulation on: every
    output equals the oracle's (search, both fusion directions, points and acceptance)."""
    w = W.make_cfg2(seed=4200, n_steps=6, forward=True)
    old = sorted(set(i for s in w["steps"] for i in s["nbrs"]) - set(s["q"] for s in w["steps"]))
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        ctx.add_keyframes(old, [w["frames"][i] for i in old])
        with ctx.server(max_batch_requests=batch, max_inflight_batches=2, tri=tm.TriParams()) as srv:
            tickets = [srv.submit(st["q"], w["frames"][st["q"]], st["nbrs"], st["q_free"], st["nbr_free"],
                                  st["mps"], fwd_mps=st["fwd_mps"], fwd_skip=st["fwd_skip"] if skip else None)
                       for st in w["steps"]]
            n_fwd = n_ok = 0
            for st, t in zip(w["steps"], tickets):
                r = srv.take_ex(t)
                assert r["info"]["status"] == 0
                exp, _ = O.search_step(w["cam"], w["frames"], st)
                assert len(r["pairs"]) == len(exp)
                for g, e in zip(r["pairs"], exp):
                    np.testing.assert_array_equal(g, e)
                fe, _ = O.fuse_step(w["cam"], w["frames"], st)
                np.testing.assert_array_equal(r["fuse"], fe)
                s2 = dict(st)
                if not skip:
                    s2["fwd_skip"] = None
                efw, _ = O.fuse_forward_step(w["cam"], w["frames"], s2)
                assert len(r["fwds"]) == len(efw)
                for g, e in zip(r["fwds"], efw):
                    np.testing.assert_array_equal(g, e)
                    n_fwd += len(e)
                off = 0
                for f, e in zip(st["nbrs"], exp):
                    xyz, ok = O.triangulate(w["cam"], w["frames"][st["q"]], w["frames"][f], e)
                    np.testing.assert_array_equal(r["points"][off:off + len(e)], xyz)
                    np.testing.assert_array_equal(r["point_ok"][off:off + len(e)], ok)
                    off += len(e)
                    n_ok += int(ok.sum())
                assert off == len(r["points"])
            assert n_fwd > 50 and n_ok > 50
