"""Pins for the oracle: each part is checked against something other than the oracle itself
(library routines, brute force, closed forms, planted geometry, hand-worked cases).

Runs on the CPU only."""

import ctypes
import json
import os

import numpy as np
import pytest

import oracle as O
from gen import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GATES_OFF = O.SearchParams(hamming_max=256, ratio_num=0, epipolar=False, resolve=False,
                           rot_filter=False)


def prefix_desc(bits):
    """Descriptors whose first `bits[k]` bits are set: Hamming(a, b) = |bits_a - bits_b|."""
    bits = np.asarray(bits, np.int64)
    out = np.zeros((len(bits), 256), np.uint8)
    for k, b in enumerate(bits):
        out[k, :b] = 1
    return np.packbits(out, axis=1)


def kf_from(desc, node, xy=None, angle=None, level=None, tcw=None):
    n = len(desc)
    return W.make_keyframe(desc, np.zeros((n, 2), np.float32) if xy is None else xy,
                           np.zeros(n, np.float32) if angle is None else angle,
                           np.zeros(n, np.uint8) if level is None else level,
                           np.asarray(node, np.uint32), np.eye(3, 4) if tcw is None else tcw,
                           -np.ones(n, np.int64))


def hamming_np(a, b):
    """All-pairs Hamming distance with numpy's bit count (library routine)."""
    x = np.bitwise_xor(a[:, None, :], b[None, :, :])
    return np.bitwise_count(x).sum(axis=2).astype(np.int64)


CAM = W.CAM_CFG0


# --------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(6))
def test_hamming_argmin_brute_force(seed):
    """Gates off, one node: every query's match is numpy's argmin of the Hamming matrix."""
    rng = np.random.default_rng(seed)
    nq, nt = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    Q = W.random_keyframe(rng, nq, CAM, n_nodes=1)
    T = W.random_keyframe(rng, nt, CAM, n_nodes=1)
    m, ncmp = O.search_pair(CAM, Q, T, params=GATES_OFF)
    D = hamming_np(Q["desc"], T["desc"])
    exp = np.stack([np.arange(nq), D.argmin(axis=1), D.min(axis=1)], axis=1)
    assert ncmp == nq * nt
    np.testing.assert_array_equal(m, exp)


@pytest.mark.parametrize("seed", range(6))
def test_node_buckets_brute_force(seed):
    """Gates off, a few nodes, random masks: the match of each free query is the argmin over
    free same-node targets; the comparison count is the size of that join."""
    rng = np.random.default_rng(100 + seed)
    nq, nt = int(rng.integers(0, 60)), int(rng.integers(0, 60))
    Q = W.random_keyframe(rng, nq, CAM, n_nodes=4)
    T = W.random_keyframe(rng, nt, CAM, n_nodes=4)
    fq = (rng.random(nq) < 0.8).astype(np.uint8)
    ft = (rng.random(nt) < 0.8).astype(np.uint8)
    m, ncmp = O.search_pair(CAM, Q, T, fq, ft, GATES_OFF)
    D = hamming_np(Q["desc"], T["desc"]) if nq and nt else np.zeros((nq, nt), np.int64)
    ok = (Q["node"][:, None] == T["node"][None, :]) & (fq[:, None] > 0) & (ft[None, :] > 0)
    assert ncmp == int(ok.sum())
    Dm = np.where(ok, D, 10 ** 6)
    rows = [(i, int(Dm[i].argmin()), int(Dm[i].min())) for i in range(nq) if ok[i].any()]
    np.testing.assert_array_equal(m.reshape(-1, 3), np.array(rows, np.int64).reshape(-1, 3))


# --------------------------------------------------------------------------- hand-worked cases

def test_ratio_golden():
    g = json.load(open(os.path.join(GOLD, "ratio_cases.json")))
    p = O.SearchParams(epipolar=False, rot_filter=False)
    for case in g["cases"]:
        d = case["dists"]
        Q = kf_from(prefix_desc([0]), [0])
        T = kf_from(prefix_desc(d) if d else np.zeros((0, 32), np.uint8), [0] * len(d))
        m, _ = O.search_pair(CAM, Q, T, params=p)
        assert m.tolist() == case["expect"], case


def test_resolve_golden():
    g = json.load(open(os.path.join(GOLD, "resolve_cases.json")))
    p = O.SearchParams(epipolar=False, rot_filter=False)
    for case in g["cases"]:
        Q = kf_from(prefix_desc(case["q_bits"]), case["q_node"])
        T = kf_from(prefix_desc(case["t_bits"]), case["t_node"])
        m, _ = O.search_pair(CAM, Q, T, params=p)
        assert m.tolist() == case["expect"], case


def test_rotation_golden():
    g = json.load(open(os.path.join(GOLD, "rotation_cases.json")))
    p = O.SearchParams(epipolar=False)
    for case in g["cases"]:
        n = len(case["q_angle"])
        qa = np.asarray(case["q_angle"], np.float32)
        ta = np.asarray(case.get("t_angle", [0.0] * n), np.float32)
        Q = kf_from(prefix_desc([0] * n), np.arange(n), angle=qa)
        T = kf_from(prefix_desc([0] * n), np.arange(n), angle=ta)
        m, _ = O.search_pair(CAM, Q, T, params=p)
        assert m[:, 0].tolist() == case["expect_q"], case
        assert (m[:, 0] == m[:, 1]).all()


def test_fuse_golden():
    g = json.load(open(os.path.join(GOLD, "fuse_cases.json")))
    cam = dict(g["camera"])
    k = g["keypoints"]
    T = kf_from(prefix_desc(k["bits"]), np.zeros(len(k["bits"])),
                xy=np.asarray(k["xy"], np.float32), level=np.asarray(k["level"], np.uint8),
                tcw=np.asarray(g["Tcw"], np.float64).reshape(3, 4))
    mp = g["mappoints"]
    n = len(mp["pos"])
    mps = dict(n=n, pos=np.asarray(mp["pos"], np.float32), normal=np.asarray(mp["normal"], np.float32),
               desc=prefix_desc(mp["bits"]), min_dist=np.asarray(mp["min_dist"], np.float32),
               max_dist=np.asarray(mp["max_dist"], np.float32), skip=np.asarray(mp["skip"], np.uint8))
    m, ncmp = O.fuse(cam, T, mps)
    assert m.tolist() == g["expect"]
    assert ncmp == g["expect_comparisons"]


# --------------------------------------------------------------------------- closed forms

def _pose_pair(rng):
    ta = W.yaw_pose(rng.normal(0, 1, 3), rng.uniform(-30, 30))
    tb = W.yaw_pose(rng.normal(0, 1, 3), rng.uniform(-30, 30))
    # add pitch/roll so that no entry of R is structurally zero
    def tilt(t, ax, ay):
        cx, sx, cy, sy = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay)
        rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
        rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
        r = rx @ rz @ t[:, :3]
        c = W.camera_center(t)
        return np.hstack([r, (-r @ c)[:, None]])
    return tilt(ta, *rng.uniform(-0.3, 0.3, 2)), tilt(tb, *rng.uniform(-0.3, 0.3, 2))


@pytest.mark.parametrize("seed", range(5))
def test_fundamental_epipolar_constraint(seed):
    """Noise-free correspondences satisfy x_Q^T F x_T = 0; the transpose does not; the
    8-point estimate (numpy SVD) of F agrees up to scale; F(T,Q) = F(Q,T)^T."""
    rng = np.random.default_rng(seed)
    tq, tt = _pose_pair(rng)
    cam = W.CAM_EUROC
    c = 0.5 * (W.camera_center(tq) + W.camera_center(tt))
    pts = c + rng.normal(0, 1, (400, 3)) + np.array([0, 0, 8.0])
    uq, vq, zq = W.project(tq, cam, pts)
    ut, vt, zt = W.project(tt, cam, pts)
    keep = (zq > 0) & (zt > 0)
    xq = np.stack([uq, vq, np.ones_like(uq)], 1)[keep]
    xt = np.stack([ut, vt, np.ones_like(ut)], 1)[keep]
    F = O.fundamental(cam, tq, tt).astype(np.float64)
    # residual as a distance to the epipolar line (pixels)
    l = xq @ F
    r = np.abs((l * xt).sum(1)) / np.hypot(l[:, 0], l[:, 1])
    assert np.max(r) < 1e-2
    lt = xq @ F.T
    rt = np.abs((lt * xt).sum(1)) / np.hypot(lt[:, 0], lt[:, 1])
    assert np.median(rt) > 1.0
    A = np.stack([np.outer(a, b).ravel() for a, b in zip(xq, xt)])
    f8 = np.linalg.svd(A)[2][-1].reshape(3, 3)
    fn, f8n = F / np.linalg.norm(F), f8 / np.linalg.norm(f8)
    if np.sum(fn * f8n) < 0:
        f8n = -f8n
    assert np.max(np.abs(fn - f8n)) < 1e-4
    F2 = O.fundamental(cam, tt, tq).astype(np.float64)
    np.testing.assert_allclose(F2, F.T, rtol=1e-5, atol=1e-7 * np.abs(F).max())


def _line_distance_geometric(cam, tq, tt, xq, xt):
    """Distance of x_T to the epipolar line of x_Q, built without F: project two points of
    the viewing ray of x_Q (depths 1 and 1000) into T and measure point-to-line distance."""
    a = W.backproject(tq, cam, xq[:, 0], xq[:, 1], np.full(len(xq), 1.0))
    b = W.backproject(tq, cam, xq[:, 0], xq[:, 1], np.full(len(xq), 1000.0))
    ua, va, _ = W.project(tt, cam, a)
    ub, vb, _ = W.project(tt, cam, b)
    dx, dy = ub - ua, vb - va
    return np.abs(dx * (xt[:, 1] - va) - dy * (xt[:, 0] - ua)) / np.hypot(dx, dy)


@pytest.mark.parametrize("seed", range(3))
def test_epipolar_gate_geometric(seed):
    """One candidate per query: the oracle keeps exactly the candidates whose geometric
    distance to the epipolar line is below sqrt(3.84)*1.2^level (ties within 1e-3 excused)."""
    rng = np.random.default_rng(seed)
    p = W.make_pair_cfg0(10 + seed, n_kp=600, n_planted=600)
    cam, Q, T = p["cam"], p["Q"], p["T"]
    iq, jt = p["planted"]
    n = len(iq)
    Qs = W.permute_keyframe(Q, iq)
    Ts = W.permute_keyframe(T, jt)
    Qs["node"] = np.arange(n, dtype=np.uint32)
    Ts["node"] = np.arange(n, dtype=np.uint32)
    # levels drawn independently in the two views, so that the sigma of the gate must come
    # from the target keypoint
    Qs["level"] = W.draw_levels(rng, n)
    Ts["level"] = W.draw_levels(rng, n)
    prm = O.SearchParams(hamming_max=256, ratio_num=0, resolve=False, rot_filter=False)
    m, _ = O.search_pair(cam, Qs, Ts, params=prm)
    passed = np.zeros(n, bool)
    passed[m[:, 0]] = True
    dist = _line_distance_geometric(cam, Q["Tcw"], T["Tcw"], Qs["xy"].astype(np.float64),
                                    Ts["xy"].astype(np.float64))
    thr = 3.84 * (1.2 ** (2 * Ts["level"].astype(np.float64)))
    ratio = dist ** 2 / thr
    expect = ratio < 1.0
    near = np.abs(ratio - 1.0) < 1e-3
    assert 0.2 < expect.mean() < 0.95
    assert np.all(passed[~near] == expect[~near])


# --------------------------------------------------------------------------- planted truth

def _epi_pass_probability(p, rng, trials=400):
    """Monte-Carlo P(epipolar pass) per planted pair from the generator's geometry with
    fresh 2-px noise in both views (float64, no F)."""
    cam, Q, T = p["cam"], p["Q"], p["T"]
    iq, jt = p["planted"]
    pts = p["points"][Q["wp"][iq]]
    uq, vq, _ = W.project(Q["Tcw"], cam, pts)
    ut, vt, _ = W.project(T["Tcw"], cam, pts)
    lvl = T["level"][jt].astype(np.float64)
    thr = 3.84 * 1.2 ** (2 * lvl)
    hits = np.zeros(len(iq))
    for _ in range(trials):
        xq = np.stack([uq + rng.normal(0, 2, len(iq)), vq + rng.normal(0, 2, len(iq))], 1)
        xt = np.stack([ut + rng.normal(0, 2, len(iq)), vt + rng.normal(0, 2, len(iq))], 1)
        d = _line_distance_geometric(cam, Q["Tcw"], T["Tcw"], xq, xt)
        hits += d ** 2 < thr
    return hits / trials


@pytest.mark.parametrize("seed", range(4))
def test_planted_recovery(seed):
    """cfg0: every accepted match is a planted pair (a random pair at Hamming <= 50 has
    probability ~1e-22), and the number recovered agrees with 0.9 * P(epipolar pass)."""
    p = W.make_pair_cfg0(seed)
    m, ncmp = O.search_pair(p["cam"], p["Q"], p["T"])
    iq, jt = p["planted"]
    planted = set(zip(iq.tolist(), jt.tolist()))
    assert all((int(a), int(b)) in planted for a, b, _ in m)
    prob = 0.9 * _epi_pass_probability(p, np.random.default_rng(99 + seed))
    mean, sd = prob.sum(), np.sqrt((prob * (1 - prob)).sum())
    assert abs(len(m) - mean) < 4.5 * sd + 3, (len(m), mean, sd)
    assert 300 < ncmp < 600  # ~ 0.9*200 + 500^2/1000


def test_permutation_invariance():
    """Relabelling the keypoints of either frame relabels the matches and nothing else."""
    p = W.make_pair_cfg0(7)
    cam, Q, T = p["cam"], p["Q"], p["T"]
    m0, c0 = O.search_pair(cam, Q, T)
    rng = np.random.default_rng(5)
    pq, pt = rng.permutation(Q["n"]), rng.permutation(T["n"])
    m1, c1 = O.search_pair(cam, W.permute_keyframe(Q, pq), W.permute_keyframe(T, pt))
    back = sorted((int(pq[a]), int(pt[b]), int(d)) for a, b, d in m1)
    assert back == sorted(map(tuple, m0.tolist()))
    assert c0 == c1


def test_step_invariants():
    """cfg1: per pair each target at most once, d == numpy Hamming <= 50, same node, masks
    respected, sorted by query, at most three rotation bins."""
    w = W.make_cfg1()
    st = w["steps"][0]
    Q = w["frames"][st["q"]]
    res, _ = O.search_step(w["cam"], w["frames"], st)
    total = 0
    for k, (f, m) in enumerate(zip(st["nbrs"], res)):
        T = w["frames"][f]
        total += len(m)
        if not len(m):
            continue
        q, t, d = m.T
        assert len(set(t.tolist())) == len(t) and np.all(np.diff(q) > 0)
        assert np.all(d <= 50)
        dd = np.bitwise_count(np.bitwise_xor(Q["desc"][q], T["desc"][t])).sum(1)
        np.testing.assert_array_equal(dd, d)
        assert np.all(Q["node"][q] == T["node"][t])
        assert np.all(st["q_free"][q] == 1) and np.all(st["nbr_free"][k][t] == 1)
        rot = np.mod(Q["angle"][q].astype(np.float64) - T["angle"][t], 360.0)
        assert len(np.unique(np.floor(rot / 12.0) % 30)) <= 3
        # planted truth: matches are the same world point
        assert np.all(Q["wp"][q] == T["wp"][t]) and np.all(Q["wp"][q] >= 0)
    assert total > 300


# --------------------------------------------------------------------------- fusion

def _fuse_geometry_f64(cam, T, mps):
    """Projection gates and predicted level in float64, written from the pinhole model."""
    R, t = T["Tcw"][:, :3], T["Tcw"][:, 3]
    pos = mps["pos"].astype(np.float64)
    pc = pos @ R.T + t
    z = pc[:, 2]
    with np.errstate(all="ignore"):
        u = cam["fx"] * pc[:, 0] / z + cam["cx"]
        v = cam["fy"] * pc[:, 1] / z + cam["cy"]
    o = W.camera_center(T["Tcw"])
    po = pos - o
    dist = np.linalg.norm(po, axis=1)
    cosv = (po * mps["normal"]).sum(1) / dist
    ok = (z > 0) & (u >= 0) & (u < cam["width"]) & (v >= 0) & (v < cam["height"])
    ok &= (dist >= mps["min_dist"]) & (dist <= mps["max_dist"]) & (cosv >= 0.5)
    with np.errstate(all="ignore"):
        pl = np.clip(np.ceil(np.log(mps["max_dist"] / dist) / np.log(1.2)), 0, 7).astype(int)
    return ok, u, v, dist, cosv, pl


def _random_mps(rng, T, cam, n):
    o = W.camera_center(T["Tcw"])
    R = T["Tcw"][:, :3]
    d = rng.uniform(1, 12, n)
    u = rng.uniform(-50, cam["width"] + 50, n)
    v = rng.uniform(-50, cam["height"] + 50, n)
    pos = W.backproject(T["Tcw"], cam, u, v, d * rng.choice([1, -1], n, p=[0.9, 0.1]))
    view = pos - o
    view /= np.linalg.norm(view, axis=1)[:, None]
    nrm = view + rng.normal(0, 0.6, (n, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    dist = np.linalg.norm(pos - o, axis=1)
    mx = dist * 1.2 ** rng.uniform(-0.5, 7.5, n)
    mn = mx / 1.2 ** 7 * rng.uniform(0.5, 1.5, n)
    return dict(n=n, pos=pos.astype(np.float32), normal=nrm.astype(np.float32),
                desc=W.random_desc(rng, n), min_dist=mn.astype(np.float32),
                max_dist=mx.astype(np.float32), skip=(rng.random(n) < 0.1).astype(np.uint8))


@pytest.mark.parametrize("seed", range(3))
def test_fuse_gates_geometric(seed):
    """With an unbounded window, chi2 and Hamming threshold, a map point yields a result
    iff it passes the projection, distance and viewing-angle gates (float64 pinhole model;
    cases within 1e-4 of a threshold excused), and the result is numpy's argmin of the
    Hamming distance over keypoints at level pl-1 or pl."""
    rng = np.random.default_rng(seed)
    cam = W.CAM_EUROC
    T = W.random_keyframe(rng, 400, cam, tcw=W.yaw_pose([0.2, 0.0, -0.1], 7.0))
    mps = _random_mps(rng, T, cam, 3000)
    m, ncmp = O.fuse(cam, T, mps, O.FuseParams(chi2=1e30, hamming_max=256, radius_scale=1e6))
    ok, u, v, dist, cosv, pl = _fuse_geometry_f64(cam, T, mps)
    ok &= mps["skip"] == 0
    with np.errstate(all="ignore"):
        lvl_f = np.log(mps["max_dist"] / dist) / np.log(1.2)
    near = ((np.abs(u) < 1e-3) | (np.abs(u - cam["width"]) < 1e-3) |
            (np.abs(v) < 1e-3) | (np.abs(v - cam["height"]) < 1e-3) |
            (np.abs(dist / mps["min_dist"] - 1) < 1e-4) | (np.abs(dist / mps["max_dist"] - 1) < 1e-4) |
            (np.abs(cosv - 0.5) < 1e-4) | (np.abs(lvl_f - np.round(lvl_f)) < 1e-4))
    got = np.zeros(mps["n"], bool)
    got[m[:, 0]] = True
    assert np.all(got[~near] == ok[~near])
    assert 0.1 < ok.mean() < 0.9
    D = hamming_np(mps["desc"], T["desc"])
    for mi, kj, d in m:
        if near[mi]:
            continue
        allowed = (T["level"] == pl[mi]) | (T["level"] == pl[mi] - 1)
        if not allowed.any():
            continue
        row = np.where(allowed, D[mi], 10 ** 6)
        assert kj == int(row.argmin()) and d == int(row.min())


def test_fuse_planted():
    """cfg1: every fusion candidate joins a map point to a keypoint of the same world point
    (a random descriptor pair at <= 50 is ~1e-22), and most fusable map points are found."""
    w = W.make_cfg1()
    st = w["steps"][0]
    Q = w["frames"][st["q"]]
    mps = st["mps"]
    m, ncmp = O.fuse_step(w["cam"], w["frames"], st)
    assert len(m) > 20
    assert np.all(mps["wp"][m[:, 0]] == Q["wp"][m[:, 1]])
    assert np.all(mps["skip"][m[:, 0]] == 0)
    assert np.all(np.diff(m[:, 0]) > 0)
    dd = np.bitwise_count(np.bitwise_xor(mps["desc"][m[:, 0]], Q["desc"][m[:, 1]])).sum(1)
    np.testing.assert_array_equal(dd, m[:, 2])


def test_forward_fusion_skip_and_independence():
    """Forward fusion (the new keyframe's map points into each neighbour): every map point is
    fused independently of the others, so with skip flags the result is exactly the rows of
    the unflagged map points in the result without flags; and a neighbour that observes every
    map point gets nothing and costs no comparisons."""
    w = W.make_cfg1(forward=True)
    st = w["steps"][0]
    fw = st["fwd_mps"]
    assert fw["n"] > 50 and len(st["fwd_skip"]) == len(st["nbrs"])
    res, ncmp = O.fuse_forward_step(w["cam"], w["frames"], st)
    assert len(res) == len(st["nbrs"]) and ncmp > 0
    some = False
    for k, f in enumerate(st["nbrs"]):
        free = dict(fw)
        free["skip"] = None
        full, _ = O.fuse(w["cam"], w["frames"][f], free)
        keep = st["fwd_skip"][k][full[:, 0]] == 0 if len(full) else np.zeros(0, bool)
        np.testing.assert_array_equal(res[k], full[keep])
        some |= bool(len(res[k]))
    assert some
    allskip = dict(st)
    allskip["fwd_skip"] = [np.ones(fw["n"], np.uint8) for _ in st["nbrs"]]
    r2, c2 = O.fuse_forward_step(w["cam"], w["frames"], allskip)
    assert c2 == 0 and all(len(x) == 0 for x in r2)


def test_orb_rotation_bins_golden():
    """ORB-family binning (rot_mode 1): nearest integer of rot * (1/30), halves away from zero,
    values worked by hand at the rounding boundaries; mode 0 keeps 30 bins of 12 degrees."""
    cases = [((15.0, 0.0), 1), ((14.99, 0.0), 0), ((45.0, 0.0), 2), ((44.9, 0.0), 1),
             ((0.0, 15.0), 12), ((0.0, 0.01), 12), ((344.9, 0.0), 11), ((0.0, 0.0), 0),
             ((100.0, 40.0), 2), ((40.0, 100.0), 10)]
    for (aq, at), b in cases:
        assert O.rot_bin(aq, at, 1) == b, (aq, at)
    assert [O.rot_bin(a, 0.0, 0) for a in (0.0, 11.99, 12.0, 359.9)] == [0, 0, 1, 29]


@pytest.mark.parametrize("seed", range(3))
def test_epipole_on_every_epipolar_line(seed):
    """The epipole in T (Q's centre projected into T) is the common point of the epipolar
    lines F^T x_Q of every query pixel: a * ex + b * ey + c = 0 up to float32 rounding.  On a
    pair whose new keyframe sits at the origin, and on pairs of a trajectory where neither
    camera does (so that the sign and origin of Q's centre matter)."""
    p = W.make_pair_cfg0(seed)
    pairs = [(p["cam"], p["Q"], p["T"])]
    w = W.make_cfg1(seed=1000 + seed)
    st = w["steps"][0]
    pairs += [(w["cam"], w["frames"][st["q"]], w["frames"][f]) for f in st["nbrs"][:3]]
    rng = np.random.default_rng(seed)
    for cam, Q, T in pairs:
        e = O.epipole(cam, Q["Tcw"], T["Tcw"]).astype(np.float64)
        F = np.zeros(9, np.float32)
        O.lib().orc_fundamental(ctypes.byref(O._cam(cam)), np.ascontiguousarray(Q["Tcw"], np.float64).ctypes.data,
                                np.ascontiguousarray(T["Tcw"], np.float64).ctypes.data, F.ctypes.data)
        F = F.astype(np.float64).reshape(3, 3)
        for _ in range(20):
            xq = np.array([rng.uniform(0, cam["width"]), rng.uniform(0, cam["height"]), 1.0])
            l = F.T @ xq
            d = abs(l[0] * e[0] + l[1] * e[1] + l[2]) / np.hypot(l[0], l[1])
            assert d < 1e-3 * max(1.0, np.hypot(*e) / 1000.0), d


def test_epipole_rejection_invariants():
    """With epipole rejection, no kept match targets a keypoint inside the rejection radius;
    the comparison count is unchanged (the distance is computed before the check); a radius
    covering the whole image keeps nothing; radius 0 is the default search."""
    w = W.make_cfg1()
    st = w["steps"][0]
    cam = w["cam"]
    Q = w["frames"][st["q"]]
    scale = [1.2 ** l for l in range(8)]
    for k, f in enumerate(st["nbrs"][:4]):
        T = w["frames"][f]
        ft = st["nbr_free"][k]
        base, c0 = O.search_pair(cam, Q, T, st["q_free"], ft)
        same, c1 = O.search_pair(cam, Q, T, st["q_free"], ft, O.SearchParams(epipole_px=0.0))
        np.testing.assert_array_equal(base, same)
        e = O.epipole(cam, Q["Tcw"], T["Tcw"])
        for px in (30.0, 300.0):
            m, c2 = O.search_pair(cam, Q, T, st["q_free"], ft, O.SearchParams(epipole_px=px))
            assert c2 == c0
            for _, t, _ in m:
                dx = np.float32(e[0] - T["xy"][t, 0]); dy = np.float32(e[1] - T["xy"][t, 1])
                assert dx * dx + dy * dy >= np.float32(px * px) * np.float32(scale[T["level"][t]])
        m, _ = O.search_pair(cam, Q, T, st["q_free"], ft, O.SearchParams(epipole_px=1e5))
        assert len(m) == 0


def test_triangulation_recovers_exact_points():
    """Noise-free planted correspondences: every planted match is accepted and its
    triangulated point is the planted world point (float32 throughout: rays from float32
    pixels and poses, the float32 closed-form midpoint of the two rays)."""
    p = W.make_pair_cfg0(5, noise_px=0.0)
    m, _ = O.search_pair(p["cam"], p["Q"], p["T"])
    xyz, ok = O.triangulate(p["cam"], p["Q"], p["T"], m)
    wq, wt = p["Q"]["wp"], p["T"]["wp"]
    planted = np.array([wq[a] >= 0 and wq[a] == wt[b] for a, b, _ in m])
    assert planted.sum() > 80
    assert ok[planted].all()
    err = np.linalg.norm(xyz[planted].astype(np.float64) - p["points"][wq[m[planted, 0]]], axis=1)
    depth = p["points"][wq[m[planted, 0]], 2]
    assert (err < 1e-3 * depth).all(), err.max()
    assert not xyz[ok == 0].any()


def test_triangulation_rejects_pure_rotation_and_scale_jumps():
    """No baseline (pure rotation): every ray pair is parallel, nothing is accepted.  A target
    keypoint moved four pyramid levels up breaks the scale consistency (1.2^4 > 1.8); one level
    keeps it."""
    p = W.make_pair_cfg0(6, noise_px=0.0, baseline=0.0)
    m, _ = O.search_pair(p["cam"], p["Q"], p["T"], params=O.SearchParams(epipolar=False))
    assert len(m) > 50
    _, ok = O.triangulate(p["cam"], p["Q"], p["T"], m)
    assert ok.sum() == 0
    p = W.make_pair_cfg0(7, noise_px=0.0)
    m, _ = O.search_pair(p["cam"], p["Q"], p["T"])
    _, ok0 = O.triangulate(p["cam"], p["Q"], p["T"], m)
    low = [k for k, (a, b, _) in enumerate(m) if ok0[k] and p["T"]["level"][b] <= 3]
    assert len(low) > 20
    for dl, expect in ((4, 0), (1, 1)):
        T = dict(p["T"])
        T["level"] = p["T"]["level"].copy()
        for k in low:
            T["level"][m[k, 1]] += dl
        _, ok = O.triangulate(p["cam"], p["Q"], T, m)
        assert (ok[low] == expect).all(), (dl, ok[low])


def _frame_at(centre, points, cam, level=0):
    """A keyframe with identity rotation at `centre` whose keypoints are the exact projections
    of `points` (world, float64); other keypoint fields are unused by triangulation."""
    c = np.asarray(centre, np.float64)
    Tcw = np.hstack([np.eye(3), -c[:, None]]).reshape(12)
    rel = np.asarray(points, np.float64) - c
    xy = np.stack([cam["fx"] * rel[:, 0] / rel[:, 2] + cam["cx"], cam["fy"] * rel[:, 1] / rel[:, 2] + cam["cy"]], 1)
    n = len(rel)
    return dict(n=n, xy=xy.astype(np.float32), level=np.full(n, level, np.uint8), Tcw=Tcw,
                desc=np.zeros((n, 32), np.uint8), angle=np.zeros(n, np.float32), node=np.zeros(n, np.uint32))


CAM_PIN = dict(width=640, height=480, fx=450.0, fy=450.0, cx=320.0, cy=240.0)


def test_triangulation_parallax_bound_alone():
    """Noise-free points 17-25 m away seen from two centres 0.3 m apart: the rays meet at the
    point, but their angle (0.7-1.0 degrees) is below the default parallax bound
    (cos 0.9998, 1.15 degrees), so nothing is accepted; with the bound at cos 0.99999
    (0.26 degrees) every point is accepted and recovered."""
    X = np.array([[0.1, 0.05, 20.0], [-0.5, 0.3, 17.0], [0.8, -0.4, 25.0], [0.0, 0.0, 18.0]])
    Q, T = _frame_at([0, 0, 0], X, CAM_PIN), _frame_at([0.3, 0, 0], X, CAM_PIN)
    ang = [np.degrees(np.arccos(np.dot(x, x - [0.3, 0, 0]) / np.linalg.norm(x) / np.linalg.norm(x - [0.3, 0, 0])))
           for x in X]
    assert all(0.6 < a < 1.14 for a in ang), ang
    m = np.array([[k, k, 0] for k in range(len(X))], np.int32)
    _, ok = O.triangulate(CAM_PIN, Q, T, m)
    assert ok.sum() == 0
    xyz, ok = O.triangulate(CAM_PIN, Q, T, m, O.TriParams(cos_parallax_max=0.99999))
    assert ok.all()
    assert (np.linalg.norm(xyz.astype(np.float64) - X, axis=1) < 0.01 * X[:, 2]).all()


def test_triangulation_point_behind_second_view():
    """Both lines pass through X = (0, 0, 5) exactly, X is in front of the first camera, and
    the second camera sits at (1, 0, 10) looking along +z, so X lies behind it: rejected
    (positive depth is required in both views).  The same point seen from (1, 0, 0), in front
    of both cameras, is accepted and recovered."""
    X = np.array([[0.0, 0.0, 5.0]])
    Q = _frame_at([0, 0, 0], X, CAM_PIN)
    m = np.array([[0, 0, 0]], np.int32)
    _, ok = O.triangulate(CAM_PIN, Q, _frame_at([1, 0, 10], X, CAM_PIN), m)
    assert ok[0] == 0
    xyz, ok = O.triangulate(CAM_PIN, Q, _frame_at([1, 0, 0], X, CAM_PIN), m)
    assert ok[0] == 1 and np.linalg.norm(xyz[0] - X[0]) < 1e-3


def test_pair_baseline_skip():
    """ORB-family pair skip: with T's median scene depth d known, the pair is not searched when
    baseline / d < ratio (the cfg0 baseline is 0.3 m: skipped for d = 40 m at ratio 0.01, kept
    for d = 20 m with the same matches as without the rule; unknown depth never skips)."""
    p = W.make_pair_cfg0(3)
    base, c0 = O.search_pair(p["cam"], p["Q"], p["T"])
    sp = O.SearchParams(baseline_min_ratio=0.01)
    m, c = O.search_pair(p["cam"], p["Q"], p["T"], params=sp, t_median_depth=40.0)
    assert len(m) == 0 and c == 0
    for d in (20.0, 0.0):
        m, c = O.search_pair(p["cam"], p["Q"], p["T"], params=sp, t_median_depth=d)
        np.testing.assert_array_equal(m, base)
        assert c == c0
