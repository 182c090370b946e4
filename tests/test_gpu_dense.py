"""Dense node blocks on the tensor cores (tcgen05, +-1 fp8 operands): queries whose BoW node
holds at least dense_min keypoints of the neighbour are compared with all of them as one
matrix product.  The results must equal the oracle's bit-exactly, like the candidate rounds'
(the dot product of two +-1 vectors is an integer <= 256 in magnitude, exact in float32)."""

import numpy as np
import pytest

import oracle as O
from gen import workloads as W

pytestmark = pytest.mark.gpu


def osp(sp):
    return O.SearchParams(sp.hamming_max, sp.ratio_num, sp.ratio_den, sp.epi_chi2, sp.epipolar,
                          sp.resolve, sp.rot_filter, sp.epipole_px, sp.rot_mode)


def load_step(tm, ctx, w, st):
    ids = [st["q"]] + list(st["nbrs"])
    ctx.add_keyframes(ids, [w["frames"][i] for i in ids])


def check_step(tm, ctx, w, st, sp):
    """Search of one step through the C ABI == the oracle, pair by pair; returns the match count."""
    got, ncmp = ctx.search(st["q"], st["nbrs"], st.get("q_free"), st.get("nbr_free"), sp)
    exp, ecmp = O.search_step(w["cam"], w["frames"], st, osp(sp))
    assert len(got) == len(exp)
    for g, e in zip(got, exp):
        np.testing.assert_array_equal(g, e)
    assert ncmp == ecmp
    return sum(len(e) for e in exp)


@pytest.fixture(scope="module")
def tm():
    import __graft_entry__ as g
    g.build()
    import paper_2511_02036_gb300 as tm
    return tm


@pytest.fixture(scope="module")
def dense_step():
    # 16 nodes, 1500 keypoints: ~94 x 94 same-node blocks; masks on
    return W.make_cfg3b(n_nbrs=6)


@pytest.mark.parametrize("dense_min", [16, 64, 100, 2000])
def test_dense_blocks_match_oracle(tm, dense_step, dense_min):
    """All blocks dense (16), most (64), some (100: one pair mixes both paths), none (2000)."""
    w = dense_step
    st = w["steps"][0]
    assert st.get("q_free") is not None and st.get("nbr_free") is not None
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        assert check_step(tm, ctx, w, st, tm.SearchParams(dense_min=dense_min)) > 100


@pytest.mark.parametrize("variant", ["gates_off", "no_epipolar", "no_ratio", "no_resolve",
                                     "no_rot", "loose_chi2", "orb_variants"])
def test_dense_parameter_variants(tm, dense_step, variant):
    sp = {"gates_off": dict(hamming_max=256, ratio_num=0, epipolar=False, resolve=False, rot_filter=False),
          "no_epipolar": dict(epipolar=False),
          "no_ratio": dict(ratio_num=0),
          "no_resolve": dict(resolve=False),
          "no_rot": dict(rot_filter=False),
          "loose_chi2": dict(epi_chi2=50.0),
          "orb_variants": dict(rot_mode=1)}[variant]
    w = dense_step
    st = w["steps"][0]
    if variant == "orb_variants":  # a radius that reaches into the image for most neighbours
        sp["epipole_px"] = float(np.median([np.hypot(*(O.epipole(w["cam"], w["frames"][st["q"]]["Tcw"],
                                                                   w["frames"][f]["Tcw"]) -
                                                       np.array([w["cam"]["cx"], w["cam"]["cy"]])))
                                            for f in st["nbrs"]]))
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        check_step(tm, ctx, w, st, tm.SearchParams(dense_min=16, **sp))


def test_dense_multi_tile_blocks(tm):
    """4 nodes: ~375 x 375 blocks, so each block spans several 128-query tiles and two
    256-keypoint column tiles; and one node so large that a block is one whole keyframe."""
    w = W.make_cfg3(seed=3600, n_nodes=4, n_nbrs=2)
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        for dmin in (16, 300):
            check_step(tm, ctx, w, st, tm.SearchParams(dense_min=dmin))
    w = W.make_cfg3(seed=3601, n_nodes=1, n_nbrs=1, n_kp=700)
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=1024) as ctx:
        load_step(tm, ctx, w, st)
        check_step(tm, ctx, w, st, tm.SearchParams(dense_min=16))


def test_dense_without_masks_and_pair_api(tm):
    w = W.make_cfg3b(seed=3502, n_nbrs=3, with_masks=False)
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        check_step(tm, ctx, w, st, tm.SearchParams(dense_min=32))
        # the per-pair form ignores dense_min
        check_step(tm, ctx, w, st, tm.SearchParams(dense_min=32, mode=tm.TM_MODE_PER_PAIR))


def test_dense_new_keyframe_in_batch(tm):
    """The new keyframe enters the store with the batch: the dense kernel reads its staged
    caller-order arrays (node ids not yet sorted), as the search kernel does."""
    w = W.make_cfg3b(seed=3503, n_nbrs=4)
    st = w["steps"][0]
    exp, ecmp = O.search_step(w["cam"], w["frames"], st)
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        ctx.add_keyframes(list(st["nbrs"]), [w["frames"][i] for i in st["nbrs"]])
        steps = [dict(kf_id=st["q"], nbrs=st["nbrs"], q_free=st.get("q_free"), nbr_free=st.get("nbr_free"))]
        res = ctx.batch_run(steps, sp=tm.SearchParams(dense_min=16), new=([st["q"]], [w["frames"][st["q"]]]))
        assert len(res.pairs) == len(exp)
        for g, e in zip(res.pairs, exp):
            np.testing.assert_array_equal(g, e)
        assert res.n_comparisons_search == ecmp


def test_dense_plan_counts_its_kernel(tm, dense_step):
    w = dense_step
    st = w["steps"][0]
    exp, ecmp = O.search_step(w["cam"], w["frames"], st)
    steps = [dict(kf_id=st["q"], nbrs=st["nbrs"], q_free=st.get("q_free"), nbr_free=st.get("nbr_free"))]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        with ctx.plan(steps, sp=tm.SearchParams(dense_min=16)) as plan:
            assert plan.info()["kernels_per_run"] == 4  # prep, dense, search, copy
            for timed in (False, True):
                plan.run(timed=timed)
                res = plan.results()
                for g, e in zip(res.pairs, exp):
                    np.testing.assert_array_equal(g, e)
                assert res.n_comparisons_search == ecmp
            ms = plan.stage_times()
            assert ms[0] > 0 and ms[4] > 0 and ms[3] > 0  # search, dense, copy


def test_dense_bounded_wait_reports_timeout(tm, dense_step):
    """The dense kernel's bounded wait on its MMA barrier runs out (test hook: a barrier that
    nothing arrives at, awaited after the MMAs completed): TM_ERR_TIMEOUT, and the context
    keeps working."""
    from paper_2511_02036_gb300 import _lib as L
    w = dense_step
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        ctx.debug_set(L.TM_DEBUG_WAIT_LIMIT, 20_000_000)
        ctx.debug_set(L.TM_DEBUG_STARVE_WAITS, 1)
        with pytest.raises(tm.TMError) as e:
            ctx.search(st["q"], st["nbrs"], st.get("q_free"), st.get("nbr_free"), tm.SearchParams(dense_min=16))
        assert e.value.status == tm.TM_ERR_TIMEOUT
        ctx.debug_set(L.TM_DEBUG_STARVE_WAITS, 0)
        check_step(tm, ctx, w, st, tm.SearchParams(dense_min=16))


def test_dense_min_validation(tm, dense_step):
    w = dense_step
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        with pytest.raises(tm.TMError) as e:
            ctx.search(st["q"], st["nbrs"], params=tm.SearchParams(dense_min=8))
        assert e.value.status == tm.TM_ERR_INVALID_ARG


def test_dense_batch_matches_oracle(tm):
    """Several cfg3b-model steps as one plan (the batched dense workload's model, fewer steps):
    dense blocks on the tensor cores for every pair of the batch, results equal the oracle's
    pair by pair, and the candidate rounds' (dense_min 0) too."""
    w = W.make_cfg3b_batch(seed=3610, n_steps=3, n_nbrs=8)
    steps = [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"))
             for s in w["steps"]]
    exp, ecmp = [], 0
    for st in w["steps"]:
        r, c = O.search_step(w["cam"], w["frames"], st)
        exp.extend(r)
        ecmp += c
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        ids = sorted(set(i for s in w["steps"] for i in [s["q"]] + list(s["nbrs"])))
        ctx.add_keyframes(ids, [w["frames"][i] for i in ids])
        for dmin in (64, 0):
            with ctx.plan(steps, sp=tm.SearchParams(dense_min=dmin)) as plan:
                plan.run()
                res = plan.results()
            assert len(res.pairs) == len(exp) and res.n_comparisons_search == ecmp
            for g, e in zip(res.pairs, exp):
                np.testing.assert_array_equal(g, e)
