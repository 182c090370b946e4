"""Seeded synthetic keyframe workloads shaped like the EuRoC / TUM-VI local-mapping steps.

Input generation only: this module draws cameras, poses, keypoints, descriptors, BoW node
ids, masks and map points.  It holds none of the matching arithmetic (no Hamming distance,
no epipolar or projection gate, no ratio test, no histogram): both the CPU oracle and the
CUDA path consume what it produces, and neither is imported here.

The real datasets (EuRoC, TUM-VI; Sec. V-A) are not available, so each workload below is a
stand-in with the camera shape, keypoint count, pyramid, descriptor-noise and vocabulary
model of the corresponding configuration:

  cfg0   one keyframe pair, 640x480 f=450, 500 kp, 200 planted pairs, 2-px noise
  cfg1   EuRoC-shaped step, 752x480 f=458, new KF + 10 neighbours, 1200 kp, 40 % shared
  cfg2   64 independent cfg1-model steps, 5..20 neighbours, 600..2000 kp per frame
  cfg3   TUM-VI-shaped step, 512x512 f=190, new KF + 20 neighbours, 1500 kp, 50 % shared,
         flip rate 0.08, 10000 nodes
  cfg3b  cfg3 with 16 nodes, so that same-node candidate blocks are dense (>= 64 x 64)
  cfg4   a stream of keyframes along a 10-minute trajectory for the serving loop

Every array is a plain numpy array.  A keyframe is a dict with keys
  desc  (n, 32) uint8   256-bit descriptor
  xy    (n, 2)  float32 pixel position
  angle (n,)    float32 orientation in degrees, [0, 360)
  level (n,)    uint8   pyramid level 0..7
  node  (n,)    uint32  BoW vocabulary node id
  Tcw   (3, 4)  float64 world -> camera pose [R | t]
  wp    (n,)    int64   world-point id of the keypoint, -1 for clutter (ground truth only)
"""

from __future__ import annotations

import numpy as np

N_LEVELS = 8
SCALE_FACTOR = 1.2
DESC_BYTES = 32


# --------------------------------------------------------------------------- cameras, poses

def camera(width, height, f, cx=None, cy=None):
    return dict(width=int(width), height=int(height), fx=float(f), fy=float(f),
                cx=float(width / 2 if cx is None else cx),
                cy=float(height / 2 if cy is None else cy))


CAM_CFG0 = camera(640, 480, 450.0, 320.0, 240.0)
CAM_EUROC = camera(752, 480, 458.0, 376.0, 240.0)
CAM_TUMVI = camera(512, 512, 190.0, 256.0, 256.0)


def yaw_pose(center, yaw_deg):
    """Tcw (3x4, float64) of a camera at `center` whose optical axis is turned by
    `yaw_deg` about the world y axis."""
    a = np.deg2rad(yaw_deg)
    ca, sa = np.cos(a), np.sin(a)
    r_wc = np.array([[ca, 0.0, sa], [0.0, 1.0, 0.0], [-sa, 0.0, ca]])
    r_cw = r_wc.T
    t = -r_cw @ np.asarray(center, dtype=np.float64)
    return np.hstack([r_cw, t[:, None]])


def camera_center(tcw):
    return -tcw[:, :3].T @ tcw[:, 3]


def project(tcw, cam, pts):
    """Pinhole projection of world points (m, 3) -> (u, v, z) in float64."""
    pc = pts @ tcw[:, :3].T + tcw[:, 3]
    z = pc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = cam["fx"] * pc[:, 0] / z + cam["cx"]
        v = cam["fy"] * pc[:, 1] / z + cam["cy"]
    return u, v, z


def backproject(tcw, cam, u, v, depth):
    xc = np.stack([(u - cam["cx"]) / cam["fx"] * depth,
                   (v - cam["cy"]) / cam["fy"] * depth, depth], axis=1)
    r_cw, t = tcw[:, :3], tcw[:, 3]
    return (xc - t) @ r_cw  # R^T (xc - t)


def in_image(cam, u, v, z):
    return (z > 0.0) & (u >= 0) & (u < cam["width"]) & (v >= 0) & (v < cam["height"])


# --------------------------------------------------------------------------- attributes

def level_probs():
    """P(level) proportional to 1.2^-level (ORB-like per-level feature allocation)."""
    w = SCALE_FACTOR ** -np.arange(N_LEVELS, dtype=np.float64)
    return w / w.sum()


def draw_levels(rng, n):
    return rng.choice(N_LEVELS, size=n, p=level_probs()).astype(np.uint8)


def random_desc(rng, n):
    return rng.integers(0, 256, size=(n, DESC_BYTES), dtype=np.uint8)


def flip_bits(rng, desc, p):
    """Each of the 256 bits flips independently with probability p."""
    if len(desc) == 0 or p <= 0:
        return desc.copy()
    bits = rng.random((len(desc), 8 * DESC_BYTES), dtype=np.float32) < p
    return desc ^ np.packbits(bits, axis=1)


def wrap_angle(a):
    a = np.mod(a, 360.0)
    a[a >= 360.0] = 0.0
    return a.astype(np.float32)


def clip_xy(cam, x, y):
    x = np.clip(x, 0.0, np.nextafter(np.float32(cam["width"]), 0))
    y = np.clip(y, 0.0, np.nextafter(np.float32(cam["height"]), 0))
    return np.stack([x, y], axis=1).astype(np.float32)


def scale_of(level):
    return SCALE_FACTOR ** np.asarray(level, dtype=np.float64)


def make_keyframe(desc, xy, angle, level, node, tcw, wp):
    n = len(desc)
    return dict(n=n,
                desc=np.ascontiguousarray(desc, dtype=np.uint8).reshape(n, DESC_BYTES),
                xy=np.ascontiguousarray(xy, dtype=np.float32).reshape(n, 2),
                angle=np.ascontiguousarray(angle, dtype=np.float32).reshape(n),
                level=np.ascontiguousarray(level, dtype=np.uint8).reshape(n),
                node=np.ascontiguousarray(node, dtype=np.uint32).reshape(n),
                Tcw=np.ascontiguousarray(tcw, dtype=np.float64).reshape(3, 4),
                wp=np.ascontiguousarray(wp, dtype=np.int64).reshape(n))


def empty_keyframe(tcw):
    return make_keyframe(np.zeros((0, 32), np.uint8), np.zeros((0, 2), np.float32),
                         np.zeros(0, np.float32), np.zeros(0, np.uint8),
                         np.zeros(0, np.uint32), tcw, np.zeros(0, np.int64))


def permute_keyframe(kf, perm):
    out = dict(kf)
    for k in ("desc", "xy", "angle", "level", "node", "wp"):
        out[k] = np.ascontiguousarray(kf[k][perm])
    return out


# --------------------------------------------------------------------------- cfg0: one pair

def make_pair_cfg0(seed, n_kp=500, n_planted=200, noise_px=2.0, flip_p=0.06,
                   n_nodes=1000, node_share=0.9, baseline=0.3, yaw_deg=5.0,
                   depth=(2.0, 10.0), cam=CAM_CFG0):
    """Single keyframe pair: planted correspondences from uniform 3D points at 2-10 m seen
    by a reference camera Q (identity pose) and a camera T displaced 0.3 m laterally and
    turned 5 deg in yaw; the remaining keypoints are uniform clutter.

    Returns dict(cam, Q, T, planted=(iQ, jT) int arrays)."""
    rng = np.random.default_rng(seed)
    tq = yaw_pose([0.0, 0.0, 0.0], 0.0)
    tt = yaw_pose([baseline, 0.0, 0.0], yaw_deg)
    pts = np.zeros((0, 3))
    uq = vq = ut = vt = np.zeros(0)
    while len(pts) < n_planted:
        m = 2 * (n_planted - len(pts)) + 16
        u = rng.uniform(0, cam["width"], m)
        v = rng.uniform(0, cam["height"], m)
        d = rng.uniform(depth[0], depth[1], m)
        p = backproject(tq, cam, u, v, d)
        u2, v2, z2 = project(tt, cam, p)
        ok = in_image(cam, u2, v2, z2)
        pts = np.vstack([pts, p[ok]])
        uq = np.concatenate([uq, u[ok]]); vq = np.concatenate([vq, v[ok]])
        ut = np.concatenate([ut, u2[ok]]); vt = np.concatenate([vt, v2[ok]])
    pts, uq, vq, ut, vt = (a[:n_planted] for a in (pts, uq, vq, ut, vt))
    n_cl = n_kp - n_planted
    lvl = draw_levels(rng, n_planted)
    base = random_desc(rng, n_planted)
    ang = rng.uniform(0, 360, n_planted)
    node_q = rng.integers(0, n_nodes, n_planted)
    node_t = np.where(rng.random(n_planted) < node_share, node_q,
                      rng.integers(0, n_nodes, n_planted))

    def frame(tcw, u, v, node, ang_p, own_seed_shift):
        xy_p = clip_xy(cam, u + rng.normal(0, noise_px, n_planted),
                       v + rng.normal(0, noise_px, n_planted))
        desc_p = flip_bits(rng, base, flip_p)
        xy_c = clip_xy(cam, rng.uniform(0, cam["width"], n_cl), rng.uniform(0, cam["height"], n_cl))
        desc = np.vstack([desc_p, random_desc(rng, n_cl)])
        xy = np.vstack([xy_p, xy_c])
        angle = np.concatenate([ang_p, rng.uniform(0, 360, n_cl)])
        level = np.concatenate([lvl, draw_levels(rng, n_cl)])
        nodes = np.concatenate([node, rng.integers(0, n_nodes, n_cl)])
        wp = np.concatenate([np.arange(n_planted), -np.ones(n_cl, np.int64)])
        kf = make_keyframe(desc, xy, wrap_angle(angle), level, nodes, tcw, wp)
        return permute_keyframe(kf, rng.permutation(n_kp))

    q = frame(tq, uq, vq, node_q, ang, 0)
    t = frame(tt, ut, vt, node_t, ang + rng.normal(0, 3.0, n_planted), 1)
    return dict(cam=cam, Q=q, T=t, planted=planted_pairs(q, t), points=pts)


def planted_pairs(q, t):
    """(iQ, jT) of keypoints that observe the same world point."""
    pos_t = {int(w): j for j, w in enumerate(t["wp"]) if w >= 0}
    iq, jt = [], []
    for i, w in enumerate(q["wp"]):
        if w >= 0 and int(w) in pos_t:
            iq.append(i); jt.append(pos_t[int(w)])
    return np.array(iq, np.int64), np.array(jt, np.int64)


# --------------------------------------------------------------------------- sequences

def trajectory(n, spacing, start=0.0, heading0=0.0, turn_deg_per_kf=0.4, look_deg=60.0):
    """KF poses along a smooth planar path: `spacing` metres between keyframes, heading
    turning slowly, the camera looking `look_deg` off the direction of travel (so that the
    motion is part lateral, part forward)."""
    poses, c = [], np.zeros(3)
    heading = np.deg2rad(heading0)
    for k in range(n):
        if k:
            c = c + spacing * np.array([np.sin(heading), 0.0, np.cos(heading)])
        heading += np.deg2rad(turn_deg_per_kf)
        poses.append(yaw_pose(c, np.rad2deg(heading) + look_deg))
    return poses


class Sequence:
    """Keyframes sharing a world-point pool.  Frame k creates `new_frac * n_shared_k` world
    points in its own view (uniform pixel, depth U[2,10] m); each point stays observable for
    a span of frames around its creator (geometric, mean `span` frames on each side).  Frame
    k's shared keypoints are a random subset of the visible pool points whose span covers k,
    and the rest of its keypoints are clutter."""

    def __init__(self, rng, cam, poses, n_kp, share, flip_p, n_nodes, node_share=0.9,
                 noise_scale_px=1.0, new_frac=0.14, span=6.0, depth=(2.0, 10.0),
                 mapped_frac=0.5):
        self.rng, self.cam, self.poses = rng, cam, poses
        nf = len(poses)
        n_kp = np.broadcast_to(np.asarray(n_kp), (nf,)).astype(np.int64)
        self.n_kp = n_kp
        n_sh = np.round(share * n_kp).astype(np.int64)
        # --- world-point pool
        created_by, pts = [], []
        for k in range(nf):
            m = int(np.ceil(new_frac * n_sh[k])) + 1
            u = rng.uniform(0, cam["width"], m)
            v = rng.uniform(0, cam["height"], m)
            d = rng.uniform(depth[0], depth[1], m)
            pts.append(backproject(poses[k], cam, u, v, d))
            created_by.append(np.full(m, k))
        self.pts = np.vstack(pts)
        self.created_by = np.concatenate(created_by)
        npool = len(self.pts)
        p_geo = 1.0 / (1.0 + span)
        span_max = 80  # geometric spans are cut at 80 frames (P > 80 is ~5e-6 at mean 6)
        self.first = self.created_by - np.minimum(rng.geometric(p_geo, npool), span_max) + 1
        self.last = self.created_by + np.minimum(rng.geometric(p_geo, npool), span_max) - 1
        order = np.argsort(self.created_by, kind="stable")
        assert np.all(order == np.arange(npool))  # created frame by frame
        self.base_desc = random_desc(rng, npool)
        self.base_node = rng.integers(0, n_nodes, npool)
        self.base_angle = rng.uniform(0, 360, npool)
        self.base_level = draw_levels(rng, npool)
        self.mapped = rng.random(npool) < mapped_frac
        # --- frames
        self.frames = []
        for k in range(nf):
            lo = np.searchsorted(self.created_by, k - span_max)
            hi = np.searchsorted(self.created_by, k + span_max, side="right")
            cand = lo + np.nonzero((self.first[lo:hi] <= k) & (self.last[lo:hi] >= k))[0]
            u, v, z = project(poses[k], cam, self.pts[cand])
            ok = in_image(cam, u, v, z)
            cand, u, v = cand[ok], u[ok], v[ok]
            sel = rng.permutation(len(cand))[: n_sh[k]]
            wp, u, v = cand[sel], u[sel], v[sel]
            ns, ncl = len(wp), int(n_kp[k] - len(wp))
            lvl = self.base_level[wp]
            sig = noise_scale_px * scale_of(lvl)
            xy_s = clip_xy(cam, u + rng.normal(0, 1, ns) * sig, v + rng.normal(0, 1, ns) * sig)
            desc_s = flip_bits(rng, self.base_desc[wp], flip_p)
            node_s = np.where(rng.random(ns) < node_share, self.base_node[wp],
                              rng.integers(0, n_nodes, ns))
            ang_s = self.base_angle[wp] + rng.normal(0, 3.0, ns)
            kf = make_keyframe(
                np.vstack([desc_s, random_desc(rng, ncl)]),
                np.vstack([xy_s, clip_xy(cam, rng.uniform(0, cam["width"], ncl),
                                         rng.uniform(0, cam["height"], ncl))]),
                wrap_angle(np.concatenate([ang_s, rng.uniform(0, 360, ncl)])),
                np.concatenate([lvl, draw_levels(rng, ncl)]),
                np.concatenate([node_s, rng.integers(0, n_nodes, ncl)]),
                poses[k],
                np.concatenate([wp, -np.ones(ncl, np.int64)]))
            self.frames.append(permute_keyframe(kf, rng.permutation(int(n_kp[k]))))

    # ------------------------------------------------------------------ one local-mapping step
    def _forward_mps(self, q, mapped_obs, nbr_mapped_w, nbr_w):
        """The new keyframe's own map points (see step) and their per-neighbour skip bytes."""
        fq = self.frames[q]
        rng = np.random.default_rng([len(self.frames), q, 0x5eed])
        wq = fq["wp"]
        new_obs = wq >= 0
        new_obs[new_obs] = ~self.mapped[wq[new_obs]]
        idx = np.nonzero(mapped_obs | new_obs)[0]
        wps, first = np.unique(wq[idx], return_index=True)
        j = idx[first]  # the first observing keypoint of each world point
        is_new = ~self.mapped[wps]
        n = len(wps)
        pos = self.pts[wps] + rng.normal(0, 0.005, (n, 3))
        c = camera_center(fq["Tcw"])
        v = pos - c
        dist = np.linalg.norm(v, axis=1)
        maxd = dist * SCALE_FACTOR ** fq["level"][j].astype(np.int64)
        mps = dict(n=n, pos=pos.astype(np.float32).reshape(n, 3),
                   normal=(v / dist[:, None]).astype(np.float32).reshape(n, 3),
                   desc=np.ascontiguousarray(fq["desc"][j]).reshape(n, DESC_BYTES),
                   min_dist=(maxd / SCALE_FACTOR ** (N_LEVELS - 1)).astype(np.float32),
                   max_dist=maxd.astype(np.float32), wp=wps)
        partner = np.full(n, -1)  # a new point's triangulation partner: the first neighbour seeing it
        for k in range(len(nbr_w) - 1, -1, -1):
            partner[np.isin(wps, nbr_w[k])] = k
        skip = [(np.where(is_new, partner == k, np.isin(wps, mw))).astype(np.uint8)
                for k, mw in enumerate(nbr_mapped_w)]
        return mps, skip

    def step(self, q, nbrs, n_mps=None, tracked_frac=0.5, with_masks=True, clutter_mp_frac=None,
             forward=False):
        """The local-mapping step of keyframe `q` against neighbour frames `nbrs`.

        Masks: a keypoint is not free for triangulation when it already has a map point.
        Neighbour keypoints of mapped world points have one; in the new keyframe half of
        them are tracked (not free, and their map point is skipped by fusion).  Clutter
        keypoints of the neighbours are lifted to single-view map points until the map-point
        batch reaches `n_mps` (default: half the neighbours' keypoints).

        Map points: position = world point + N(0, 5 mm); descriptor = that of its first
        observing neighbour; normal = mean unit viewing direction over observing neighbours;
        maxDist = distance to the first observer * 1.2^level, minDist = maxDist / 1.2^7.

        forward=True adds the new keyframe's own map points as fwd_mps: one per world point
        it observes that is either mapped (tracked) or shared but not yet mapped (as if just
        triangulated from this step's matches), from its first keypoint of that point:
        position + N(0, 5 mm), that keypoint's descriptor, the unit direction from the new
        keyframe's centre, maxDist = distance * 1.2^level.  Per neighbour, fwd_skip is 1 where
        the neighbour already observes the point: for a mapped point, any neighbour with a
        keypoint of it; for a new point, its triangulation partner (the first neighbour with
        a keypoint of it).  Drawn from a stream of their own, so the rest of the step is the
        same with or without them."""
        rng = self.rng
        fq = self.frames[q]
        q_wp = fq["wp"]
        mq = q_wp >= 0
        mq[mq] = self.mapped[q_wp[mq]]
        tracked = np.zeros(fq["n"], bool)
        tracked[mq] = rng.random(int(mq.sum())) < tracked_frac
        tracked_wp = np.unique(q_wp[tracked])
        q_free = (~tracked).astype(np.uint8)
        nbr_has, obs_w, obs_k, obs_j, clutter, nbr_mapped_w, nbr_w = [], [], [], [], [], [], []
        for k_nb, f in enumerate(nbrs):
            fr = self.frames[f]
            w = fr["wp"]
            has = np.zeros(fr["n"], bool)
            pool_idx = np.nonzero(w >= 0)[0]
            sel = pool_idx[self.mapped[w[pool_idx]]]
            has[sel] = True
            nbr_mapped_w.append(w[sel])
            nbr_w.append(w[w >= 0])
            obs_w.append(w[sel]); obs_k.append(np.full(len(sel), k_nb)); obs_j.append(sel)
            clutter.append(np.nonzero(w < 0)[0])
            nbr_has.append(has)
        nn = len(nbrs)
        obs_w = np.concatenate(obs_w) if nn else np.zeros(0, np.int64)
        obs_k = np.concatenate(obs_k) if nn else np.zeros(0, np.int64)  # index into nbrs
        obs_j = np.concatenate(obs_j) if nn else np.zeros(0, np.int64)
        uw, first = np.unique(obs_w, return_index=True)
        n_pool = len(uw)
        if n_mps is None:
            n_mps = int(0.5 * sum(self.frames[f]["n"] for f in nbrs))
        total_clutter = sum(len(c) for c in clutter)
        frac = 0.0 if total_clutter == 0 else min(1.0, max(0, n_mps - n_pool) / total_clutter)
        if clutter_mp_frac is not None:
            frac = clutter_mp_frac
        centers = {f: camera_center(self.frames[f]["Tcw"]) for f in nbrs}
        carr = np.array([centers[f] for f in nbrs]).reshape(nn, 3)
        # pool map points
        pos_p = self.pts[uw] + rng.normal(0, 0.005, (n_pool, 3))
        ref_k, ref_j = obs_k[first], obs_j[first]
        # each pool point's reference keypoint (its first observing neighbour), gathered per
        # neighbour
        desc_p = np.zeros((n_pool, DESC_BYTES), np.uint8)
        lvl_ref = np.zeros(n_pool, np.int64)
        for k_nb in np.unique(ref_k):
            m = ref_k == k_nb
            fr = self.frames[nbrs[k_nb]]
            desc_p[m] = fr["desc"][ref_j[m]]
            lvl_ref[m] = fr["level"][ref_j[m]]
        slot = np.searchsorted(uw, obs_w)
        cobs = carr[obs_k] if len(obs_k) else np.zeros((0, 3))
        v = pos_p[slot] - cobs
        v /= np.linalg.norm(v, axis=1)[:, None]
        acc = np.zeros((n_pool, 3))
        np.add.at(acc, slot, v)
        nrm_p = acc / np.linalg.norm(acc, axis=1)[:, None] if n_pool else acc
        cref = carr[ref_k] if n_pool else np.zeros((0, 3))
        maxd_p = np.linalg.norm(pos_p - cref, axis=1) * SCALE_FACTOR ** lvl_ref
        skip_p = np.isin(uw, tracked_wp).astype(np.uint8)
        # single-view map points lifted from neighbour clutter
        pos_c, desc_c, nrm_c, maxd_c = [], [], [], []
        for f, idx, has in zip(nbrs, clutter, nbr_has):
            if frac <= 0 or len(idx) == 0:
                continue
            take = idx[rng.random(len(idx)) < frac]
            fr = self.frames[f]
            has[take] = True
            d = rng.uniform(2.0, 10.0, len(take))
            p = backproject(fr["Tcw"], self.cam, fr["xy"][take, 0].astype(np.float64),
                            fr["xy"][take, 1].astype(np.float64), d)
            nv = p - centers[f]
            dist = np.linalg.norm(nv, axis=1)
            pos_c.append(p); desc_c.append(fr["desc"][take]); nrm_c.append(nv / dist[:, None])
            maxd_c.append(dist * SCALE_FACTOR ** fr["level"][take].astype(np.int64))
        nc = sum(len(x) for x in pos_c)
        cat = lambda xs, shape: np.concatenate(xs) if xs else np.zeros(shape)  # noqa: E731
        pos = np.concatenate([pos_p, cat(pos_c, (0, 3))])
        nm = len(pos)
        maxd = np.concatenate([maxd_p, cat(maxd_c, (0,))])
        mps = dict(n=nm,
                   pos=pos.astype(np.float32).reshape(nm, 3),
                   normal=np.concatenate([nrm_p, cat(nrm_c, (0, 3))]).astype(np.float32).reshape(nm, 3),
                   desc=np.concatenate([desc_p, cat(desc_c, (0, DESC_BYTES)).astype(np.uint8)]).reshape(nm, DESC_BYTES),
                   min_dist=(maxd / SCALE_FACTOR ** (N_LEVELS - 1)).astype(np.float32),
                   max_dist=maxd.astype(np.float32),
                   skip=np.concatenate([skip_p, np.zeros(nc, np.uint8)]),
                   wp=np.concatenate([uw, -np.ones(nc, np.int64)]))
        if nm:
            perm = rng.permutation(nm)
            for k in ("pos", "normal", "desc", "min_dist", "max_dist", "skip", "wp"):
                mps[k] = np.ascontiguousarray(mps[k][perm])
        step = dict(q=q, nbrs=list(nbrs), mps=mps)
        if forward:
            step["fwd_mps"], step["fwd_skip"] = self._forward_mps(q, mq, nbr_mapped_w, nbr_w)
        if with_masks:
            step["q_free"] = q_free
            step["nbr_free"] = [(~h).astype(np.uint8) for h in nbr_has]
        else:
            step["q_free"] = None
            step["nbr_free"] = None
        return step


# --------------------------------------------------------------------------- configurations

def make_step_workload(seed, cam, n_nbrs, n_kp, share, flip_p, n_nodes, n_mps=None,
                       spacing=0.125, with_masks=True, noise_scale_px=1.0, forward=False):
    """One local-mapping step: the new keyframe is the last frame of a short trajectory and
    its covisible neighbours are the `n_nbrs` frames before it."""
    rng = np.random.default_rng(seed)
    nf = n_nbrs + 1
    poses = trajectory(nf, spacing, heading0=rng.uniform(0, 360))
    n_kp_arr = n_kp if np.ndim(n_kp) else np.full(nf, n_kp)
    seq = Sequence(rng, cam, poses, n_kp_arr, share, flip_p, n_nodes,
                   noise_scale_px=noise_scale_px)
    q = nf - 1
    nbrs = list(range(q - 1, -1, -1))
    step = seq.step(q, nbrs, n_mps=n_mps, with_masks=with_masks, forward=forward)
    return dict(cam=cam, frames=seq.frames, steps=[step])


def make_cfg1(seed=1000, with_masks=True, scale=1.0, forward=False):
    return make_step_workload(seed, CAM_EUROC, 10, int(1200 * scale), 0.4, 0.06, 1000,
                              n_mps=int(6000 * scale), with_masks=with_masks, forward=forward)


def make_cfg3(seed=3000, n_nodes=10000, with_masks=True, n_nbrs=20, n_kp=1500):
    return make_step_workload(seed, CAM_TUMVI, n_nbrs, n_kp, 0.5, 0.08, n_nodes,
                              with_masks=with_masks)


def make_cfg3b(seed=3500, **kw):
    return make_cfg3(seed=seed, n_nodes=16, **kw)


def make_cfg2(seed=2000, n_steps=64, nbr_range=(5, 20), kp_range=(600, 2000),
              with_masks=True, forward=False):
    """Independent local-mapping steps with uneven neighbour and keypoint counts, all with
    the cfg1 camera, descriptor and vocabulary model.  Frames of all steps are numbered
    consecutively in one `frames` list."""
    rng = np.random.default_rng(seed)
    frames, steps = [], []
    for s in range(n_steps):
        nn = int(rng.integers(nbr_range[0], nbr_range[1] + 1))
        nkp = rng.integers(kp_range[0], kp_range[1] + 1, nn + 1)
        sub = np.random.default_rng(int(rng.integers(1 << 62)))
        poses = trajectory(nn + 1, 0.125, heading0=sub.uniform(0, 360))
        seq = Sequence(sub, CAM_EUROC, poses, nkp, 0.4, 0.06, 1000)
        q = nn
        st = seq.step(q, list(range(q - 1, -1, -1)), with_masks=with_masks, forward=forward)
        base = len(frames)
        frames.extend(seq.frames)
        st["q"] += base
        st["nbrs"] = [b + base for b in st["nbrs"]]
        steps.append(st)
    return dict(cam=CAM_EUROC, frames=frames, steps=steps)


def make_cfg3b_batch(seed=3600, n_steps=64, n_nbrs=20, n_kp=1500, n_nodes=16, with_masks=True):
    """Independent cfg3b-model local-mapping steps (TUM-VI camera, new keyframe + n_nbrs
    neighbours, n_kp keypoints, 50 % shared points, flip rate 0.08, n_nodes BoW nodes, so that
    every node is a dense block of ~n_kp / n_nodes keypoints), as one batch.  Frames of all
    steps are numbered consecutively in one `frames` list."""
    rng = np.random.default_rng(seed)
    frames, steps = [], []
    for s in range(n_steps):
        sub = np.random.default_rng(int(rng.integers(1 << 62)))
        poses = trajectory(n_nbrs + 1, 0.125, heading0=sub.uniform(0, 360))
        seq = Sequence(sub, CAM_TUMVI, poses, np.full(n_nbrs + 1, n_kp), 0.5, 0.08, n_nodes)
        q = n_nbrs
        st = seq.step(q, list(range(q - 1, -1, -1)), with_masks=with_masks)
        base = len(frames)
        frames.extend(seq.frames)
        st["q"] += base
        st["nbrs"] = [b + base for b in st["nbrs"]]
        steps.append(st)
    return dict(cam=CAM_TUMVI, frames=frames, steps=steps)


def make_stream_cfg4(seed=4000, n_kf=3000, kp_range=(1000, 2000), nbr_range=(5, 20),
                     duration_s=600.0, with_masks=True, rate_hz=None):
    """A keyframe stream along one long trajectory.  Keyframe k's neighbours are the
    preceding min(k, U{5..20}) keyframes; arrivals are Poisson at `rate_hz` if given."""
    rng = np.random.default_rng(seed)
    spacing = 0.5 * duration_s / n_kf  # 0.5 m/s
    poses = trajectory(n_kf, spacing, heading0=rng.uniform(0, 360), turn_deg_per_kf=0.15)
    nkp = rng.integers(kp_range[0], kp_range[1] + 1, n_kf)
    seq = Sequence(rng, CAM_EUROC, poses, nkp, 0.4, 0.06, 1000)
    steps = []
    for k in range(n_kf):
        nn = min(k, int(rng.integers(nbr_range[0], nbr_range[1] + 1)))
        steps.append(seq.step(k, list(range(k - 1, k - 1 - nn, -1)), with_masks=with_masks))
    arrivals = None
    if rate_hz:
        arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n_kf))
    return dict(cam=CAM_EUROC, frames=seq.frames, steps=steps, arrivals=arrivals)


def random_keyframe(rng, n, cam, n_nodes=1000, tcw=None):
    """Unstructured keyframe: uniform everything (edge-case and fuzz tests)."""
    if tcw is None:
        tcw = yaw_pose(rng.normal(0, 0.2, 3), rng.uniform(-10, 10))
    return make_keyframe(random_desc(rng, n),
                         clip_xy(cam, rng.uniform(0, cam["width"], n), rng.uniform(0, cam["height"], n)),
                         wrap_angle(rng.uniform(0, 360, n)), draw_levels(rng, n),
                         rng.integers(0, max(1, n_nodes), n), tcw, -np.ones(n, np.int64))
