"""GPU path == oracle, element by element, on the same seeded inputs (bit-exact: the matches
are integers and every floating-point gate decision is taken in float32 on both sides by the
same expression).  All calls go through the C ABI via the Python binding."""

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
    """Oracle parameters of a binding SearchParams."""
    return O.SearchParams(sp.hamming_max, sp.ratio_num, sp.ratio_den, sp.epi_chi2, sp.epipolar,
                          sp.resolve, sp.rot_filter, sp.epipole_px, sp.rot_mode)


def ofp(fp):
    return O.FuseParams(fp.chi2, fp.hamming_max, fp.radius_scale)


def check_pair(ctx, cam, Q, T, qid, tid, sp, free_q=None, free_t=None):
    got, ncmp = ctx.search(qid, [tid], free_q, None if free_t is None else [free_t], sp)
    exp, ecmp = O.search_pair(cam, Q, T, free_q, free_t, osp(sp))
    np.testing.assert_array_equal(got[0], exp)
    assert ncmp == ecmp
    return exp


# --------------------------------------------------------------------------- cfg0: one pair

@pytest.mark.parametrize("seed", range(4))
def test_cfg0_pair(tm, seed):
    p = W.make_pair_cfg0(seed)
    with tm.Context(p["cam"], max_kp=512) as ctx:
        ctx.add_keyframes([1, 2], [p["Q"], p["T"]])
        exp = check_pair(ctx, p["cam"], p["Q"], p["T"], 1, 2, tm.SearchParams())
        assert len(exp) > 80


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("mode", [0, 1])
def test_lanes_and_modes(tm, lanes, mode):
    """Every lanes-per-query instance in both forms (batched pipeline, plain per-pair)."""
    p = W.make_pair_cfg0(11, n_nodes=40)  # denser buckets: several candidates per query
    with tm.Context(p["cam"], max_kp=512) as ctx:
        ctx.add_keyframes([1, 2], [p["Q"], p["T"]])
        check_pair(ctx, p["cam"], p["Q"], p["T"], 1, 2,
                   tm.SearchParams(lanes_per_query=lanes, mode=mode))


@pytest.mark.parametrize("variant", ["gates_off", "no_ratio", "no_epipolar", "no_resolve",
                                     "no_rot", "tight", "loose_chi2", "epipole_10", "epipole_half",
                                     "orb_bins", "orb_all"])
def test_parameter_variants(tm, variant):
    sp = {"gates_off": tm.SearchParams(hamming_max=256, ratio_num=0, epipolar=False, resolve=False,
                                       rot_filter=False),
          "no_ratio": tm.SearchParams(ratio_num=0),
          "no_epipolar": tm.SearchParams(epipolar=False),
          "no_resolve": tm.SearchParams(resolve=False),
          "no_rot": tm.SearchParams(rot_filter=False),
          "tight": tm.SearchParams(hamming_max=30, ratio_num=1, ratio_den=2),
          "loose_chi2": tm.SearchParams(epi_chi2=50.0),
          "epipole_10": tm.SearchParams(epipole_px=10.0),
          "epipole_half": tm.SearchParams(),
          "orb_bins": tm.SearchParams(rot_mode=1),
          "orb_all": tm.SearchParams.orb_family(coarse=True, baseline_min_ratio=0.0)}[variant]
    p = W.make_pair_cfg0(21, n_nodes=30)
    if variant in ("epipole_half", "orb_all"):
        # a radius reaching the image centre: the epipole of this lateral motion lies far
        # outside the image, and about half of the image is rejected
        e = O.epipole(p["cam"], p["Q"]["Tcw"], p["T"]["Tcw"])
        sp.epipole_px = float(np.hypot(e[0] - p["cam"]["cx"], e[1] - p["cam"]["cy"]))
    rng = np.random.default_rng(3)
    fq = (rng.random(p["Q"]["n"]) < 0.9).astype(np.uint8)
    ft = (rng.random(p["T"]["n"]) < 0.9).astype(np.uint8)
    with tm.Context(p["cam"], max_kp=512) as ctx:
        ctx.add_keyframes([1, 2], [p["Q"], p["T"]])
        for mode in (0, 1):
            sp.mode = mode
            check_pair(ctx, p["cam"], p["Q"], p["T"], 1, 2, sp, fq, ft)


# --------------------------------------------------------------------------- steps

def load_step(tm, ctx, w, st):
    ids = [st["q"]] + list(st["nbrs"])
    ctx.add_keyframes(ids, [w["frames"][i] for i in ids])


def check_step(tm, ctx, w, st, sp=None, fp=None):
    sp = sp or tm.SearchParams()
    fp = fp or tm.FuseParams()
    got, ncmp = ctx.search(st["q"], st["nbrs"], st.get("q_free"), st.get("nbr_free"), sp)
    exp, ecmp = O.search_step(w["cam"], w["frames"], st, osp(sp))
    assert len(got) == len(exp)
    for g, e in zip(got, exp):
        np.testing.assert_array_equal(g, e)
    assert ncmp == ecmp
    if st.get("mps") is not None:
        fg, fcmp = ctx.fuse(st["q"], st["mps"], fp)
        fe, fecmp = O.fuse_step(w["cam"], w["frames"], st, ofp(fp))
        np.testing.assert_array_equal(fg, fe)
        assert fcmp == fecmp
    return sum(len(e) for e in exp)


@pytest.mark.parametrize("masks", [True, False])
def test_cfg1_step(tm, masks):
    w = W.make_cfg1(with_masks=masks)
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        assert check_step(tm, ctx, w, st) > 300


def test_cfg3_tumvi_step(tm):
    w = W.make_cfg3()
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        assert check_step(tm, ctx, w, st) > 500


def test_cfg3b_dense_buckets(tm):
    """16 nodes: ~94 x 94 same-node blocks, many candidates per query."""
    w = W.make_cfg3b(n_nbrs=6)
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        for lanes in (1, 8, 32):
            for mode in (0, 1):
                check_step(tm, ctx, w, st, tm.SearchParams(lanes_per_query=lanes, mode=mode))


def test_fuse_variants(tm):
    w = W.make_cfg1(seed=1001)
    st = w["steps"][0]
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        Q = w["frames"][st["q"]]
        for fp in (tm.FuseParams(), tm.FuseParams(radius_scale=20.0, chi2=100.0),
                   tm.FuseParams(hamming_max=256, radius_scale=1e4, chi2=1e30)):
            fg, fcmp = ctx.fuse(st["q"], st["mps"], fp)
            fe, fecmp = O.fuse(w["cam"], Q, st["mps"], ofp(fp))
            np.testing.assert_array_equal(fg, fe)
            assert fcmp == fecmp


# --------------------------------------------------------------------------- edge cases

def test_edge_cases(tm):
    cam = W.CAM_CFG0
    rng = np.random.default_rng(7)
    kfs = {
        1: W.random_keyframe(rng, 0, cam),                 # empty
        2: W.random_keyframe(rng, 1, cam, n_nodes=1),      # single keypoint
        3: W.random_keyframe(rng, 37, cam, n_nodes=1),     # one bucket, ragged size
        4: W.random_keyframe(rng, 1000, cam, n_nodes=3),   # few huge buckets
        5: W.random_keyframe(rng, 999, cam, n_nodes=100000),  # no shared buckets
        6: W.random_keyframe(rng, 4096, cam, n_nodes=50),  # at max_kp
    }
    kfs[4]["desc"][500:520] = kfs[6]["desc"][:20]          # some real matches
    # at the largest capacity used here, and at a smaller one (ragged sizes 0, 1, 37, 999, 1000)
    for subset, cap in ((list(kfs), 4096), ([1, 2, 3, 4, 5], 1024)):
        with tm.Context(cam, max_kp=cap) as ctx:
            ctx.add_keyframes(subset, [kfs[i] for i in subset])
            for q in subset:
                nb = [t for t in subset if t != q]
                for sp in (tm.SearchParams(), tm.SearchParams(hamming_max=256, ratio_num=0, rot_filter=False)):
                    got, ncmp = ctx.search(q, nb, params=sp)
                    ecmp = 0
                    for t, g in zip(nb, got):
                        e, c = O.search_pair(cam, kfs[q], kfs[t], params=osp(sp))
                        np.testing.assert_array_equal(g, e)
                        ecmp += c
                    assert ncmp == ecmp
    with tm.Context(cam, max_kp=4096) as ctx:
        ctx.add_keyframes(list(kfs), list(kfs.values()))
        # all-zero masks: nothing to match
        got, ncmp = ctx.search(4, [6], np.zeros(1000, np.uint8), None)
        assert ncmp == 0 and len(got[0]) == 0
        # zero neighbours, zero map points
        got, ncmp = ctx.search(4, [])
        assert got == [] and ncmp == 0
        empty = dict(n=0, pos=np.zeros((0, 3), np.float32), normal=np.zeros((0, 3), np.float32),
                     desc=np.zeros((0, 32), np.uint8), min_dist=np.zeros(0, np.float32),
                     max_dist=np.zeros(0, np.float32), skip=None)
        fg, fc = ctx.fuse(6, empty)
        assert len(fg) == 0 and fc == 0


def test_device_resident_inputs(tm):
    """Keyframes, masks and map points given as CUDA tensors (device pointers)."""
    torch = pytest.importorskip("torch")
    w = W.make_cfg1(seed=1002, scale=0.5)
    st = w["steps"][0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        ids = [st["q"]] + st["nbrs"]
        dkfs = []
        for i in ids:
            f = w["frames"][i]
            dkfs.append(dict(desc=dev(f["desc"]), xy=dev(f["xy"]), angle=dev(f["angle"]),
                             level=dev(f["level"]), node=dev(f["node"].view(np.int32)), Tcw=f["Tcw"]))
        ctx.add_keyframes(ids, dkfs)
        got, ncmp = ctx.search(st["q"], st["nbrs"], dev(st["q_free"]),
                               dev(np.concatenate(st["nbr_free"])))
        exp, ecmp = O.search_step(w["cam"], w["frames"], st)
        for g, e in zip(got, exp):
            np.testing.assert_array_equal(g, e)
        mps = {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in st["mps"].items() if k != "wp"}
        fg, _ = ctx.fuse(st["q"], mps)
        fe, _ = O.fuse_step(w["cam"], w["frames"], st)
        np.testing.assert_array_equal(fg, fe)


@pytest.mark.parametrize("mode", [0, 1])
def test_orb_variants_step(tm, mode):
    """ORB-family variants on a whole EuRoC-shaped step (batched and per-pair forms): epipole
    rejection with a radius that removes matches, and the ORB rotation binning."""
    w = W.make_cfg1(seed=1003)
    st = w["steps"][0]
    d = [np.hypot(*(O.epipole(w["cam"], w["frames"][st["q"]]["Tcw"], w["frames"][f]["Tcw"]) -
                    np.array([w["cam"]["cx"], w["cam"]["cy"]]))) for f in st["nbrs"]]
    px = float(np.median(d))  # reaches the image centre for half of the neighbours
    with tm.Context(w["cam"], max_kp=2048) as ctx:
        load_step(tm, ctx, w, st)
        for sp in (tm.SearchParams(epipole_px=px, mode=mode), tm.SearchParams(rot_mode=1, mode=mode),
                   tm.SearchParams(epipole_px=px, rot_mode=1, mode=mode, lanes_per_query=4)):
            got, ncmp = ctx.search(st["q"], st["nbrs"], st.get("q_free"), st.get("nbr_free"), sp)
            exp, ecmp = O.search_step(w["cam"], w["frames"], st, osp(sp))
            for g, e in zip(got, exp):
                np.testing.assert_array_equal(g, e)
            assert ncmp == ecmp
