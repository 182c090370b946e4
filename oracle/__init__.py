"""Oracle for the correspondence search (Sec. IV-C), the fusion search (Sec. IV-D), the
triangulation checks of Map Point Creation (Sec. III), the keyframe-culling redundancy test
(Sec. IV-F) and the sequential fuse-apply stage (Sec. IV-D).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-correct CPU definition (C, in
`tm_oracle.c`; the culling test and the fuse-apply map in plain Python below) plus this ctypes
wrapper.  Only the tests, the smoke check and the benchmark's CPU-baseline / reference arm
load it; the library never does, and it shares no code with the CUDA path.

Parity pins: tests/test_oracle_pins.py (brute force, closed forms, planted geometry,
hand-worked golden cases under tests/golden/), tests/test_oracle_mutations.py (planted
mistakes caught), tests/test_fuse_apply.py (a hand-worked fuse-apply and culling case, the
map's consistency invariants).  Unpinned beyond hand-worked cases: the exact 3:5 ratio tie and
the rotation-bin boundaries (readings, not facts of the paper).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force=False, src=_SRC, out=_LIB):
    """Compile the oracle with gcc (no FMA contraction, IEEE float)."""
    hdr = os.path.join(_HERE, "tm_oracle.h")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(src), os.path.getmtime(hdr)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", *CFLAGS, "-I", _HERE, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


class _Keyframe(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32),
                ("desc", ctypes.c_void_p), ("xy", ctypes.c_void_p),
                ("angle", ctypes.c_void_p), ("level", ctypes.c_void_p),
                ("node", ctypes.c_void_p), ("Tcw", ctypes.c_double * 12)]


class _SearchParams(ctypes.Structure):
    _fields_ = [("hamming_max", ctypes.c_int32), ("ratio_num", ctypes.c_int32),
                ("ratio_den", ctypes.c_int32), ("epi_chi2", ctypes.c_float),
                ("epipolar", ctypes.c_int32), ("resolve", ctypes.c_int32),
                ("rot_filter", ctypes.c_int32), ("epipole_px", ctypes.c_float),
                ("rot_mode", ctypes.c_int32), ("baseline_min_ratio", ctypes.c_float),
                ("t_median_depth", ctypes.c_float)]


class _FuseParams(ctypes.Structure):
    _fields_ = [("chi2", ctypes.c_float), ("hamming_max", ctypes.c_int32),
                ("radius_scale", ctypes.c_float)]


@dataclass
class SearchParams:
    hamming_max: int = 50
    ratio_num: int = 3
    ratio_den: int = 5
    epi_chi2: float = 3.84
    epipolar: bool = True
    resolve: bool = True
    rot_filter: bool = True
    epipole_px: float = 0.0   # ORB-family epipole rejection radius at level 0 (0 = off)
    rot_mode: int = 0         # 0: 30 bins of 12 degrees; 1: ORB-family round(rot / 30)
    baseline_min_ratio: float = 0.0  # ORB-family pair skip: baseline / median depth below this


@dataclass
class TriParams:
    cos_parallax_max: float = 0.9998
    chi2: float = 5.991
    ratio_factor: float = 1.5 * 1.2


class _TriParams(ctypes.Structure):
    _fields_ = [("cos_parallax_max", ctypes.c_double), ("chi2", ctypes.c_double),
                ("ratio_factor", ctypes.c_double)]


@dataclass
class FuseParams:
    chi2: float = 5.99
    hamming_max: int = 50
    radius_scale: float = 3.0


_lib = None


def use_library(path):
    """Load the oracle from another build of tm_oracle.c (None: the default build).  Used by
    the mutation test, which compiles deliberately broken copies of the source."""
    global _lib
    _lib = None
    return lib(path)


def lib(path=None):
    global _lib
    if _lib is None:
        L = ctypes.CDLL(path or build())
        P = ctypes.c_void_p
        L.orc_fundamental.argtypes = [ctypes.POINTER(_Camera), P, P, P]
        L.orc_fundamental.restype = None
        L.orc_search_pair.argtypes = [ctypes.POINTER(_Camera), ctypes.POINTER(_Keyframe),
                                      ctypes.POINTER(_Keyframe), P, P,
                                      ctypes.POINTER(_SearchParams), P, P, P,
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.orc_search_pair.restype = ctypes.c_int64
        L.orc_epipole.argtypes = [ctypes.POINTER(_Camera), P, P, P]
        L.orc_epipole.restype = None
        L.orc_rot_bin_mode.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int]
        L.orc_rot_bin_mode.restype = ctypes.c_int
        L.orc_triangulate.argtypes = [ctypes.POINTER(_Camera), ctypes.POINTER(_Keyframe),
                                      ctypes.POINTER(_Keyframe), ctypes.c_int64, P, P,
                                      ctypes.POINTER(_TriParams), P, P]
        L.orc_triangulate.restype = None
        L.orc_fuse.argtypes = [ctypes.POINTER(_Camera), ctypes.POINTER(_Keyframe),
                               ctypes.c_int32, P, P, P, P, P, P,
                               ctypes.POINTER(_FuseParams), P, P, P, ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_int64)]
        L.orc_fuse.restype = ctypes.c_int64
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _cam(cam):
    return _Camera(int(cam["width"]), int(cam["height"]), float(cam["fx"]), float(cam["fy"]),
                   float(cam["cx"]), float(cam["cy"]))


def _kf(kf, keep):
    arrs = [np.ascontiguousarray(kf["desc"], np.uint8), np.ascontiguousarray(kf["xy"], np.float32),
            np.ascontiguousarray(kf["angle"], np.float32), np.ascontiguousarray(kf["level"], np.uint8),
            np.ascontiguousarray(kf["node"], np.uint32)]
    keep.extend(arrs)
    s = _Keyframe()
    s.n = int(len(arrs[0]))
    s.desc, s.xy, s.angle, s.level, s.node = (a.ctypes.data for a in arrs)
    s.Tcw[:] = [float(x) for x in np.asarray(kf["Tcw"], np.float64).reshape(12)]
    return s


def fundamental(cam, tcw_q, tcw_t):
    F = np.zeros(9, np.float32)
    a = np.ascontiguousarray(tcw_q, np.float64).reshape(12)
    b = np.ascontiguousarray(tcw_t, np.float64).reshape(12)
    c = _cam(cam)
    lib().orc_fundamental(ctypes.byref(c), a.ctypes.data, b.ctypes.data, F.ctypes.data)
    return F.reshape(3, 3)


def _mask(m):
    return None if m is None else np.ascontiguousarray(m, np.uint8)


def epipole(cam, Tq, Tt):
    """The epipole in T (float32 pair): Q's camera centre projected into T."""
    c = _cam(cam)
    q = np.ascontiguousarray(Tq, np.float64).reshape(12)
    t = np.ascontiguousarray(Tt, np.float64).reshape(12)
    e = np.zeros(2, np.float32)
    lib().orc_epipole(ctypes.byref(c), q.ctypes.data, t.ctypes.data, e.ctypes.data)
    return e


def rot_bin(angle_q, angle_t, mode=0):
    """Rotation-histogram bin of a match under rot_mode `mode`."""
    return int(lib().orc_rot_bin_mode(float(angle_q), float(angle_t), int(mode)))


def triangulate(cam, Q, T, matches, params=None):
    """Triangulation of a pair's matches (k, 3) int32 (q_idx, t_idx, dist) and their
    acceptance as new map points: float32 (k, 3) points (0 where rejected) and uint8 (k,) flags."""
    p = params or TriParams()
    keep = []
    q, t = _kf(Q, keep), _kf(T, keep)
    m = np.ascontiguousarray(np.asarray(matches, np.int32).reshape(-1, 3))
    qi, ti = np.ascontiguousarray(m[:, 0]), np.ascontiguousarray(m[:, 1])
    xyz = np.zeros((len(m), 3), np.float32)
    ok = np.zeros(len(m), np.uint8)
    tp = _TriParams(p.cos_parallax_max, p.chi2, p.ratio_factor)
    lib().orc_triangulate(ctypes.byref(_cam(cam)), ctypes.byref(q), ctypes.byref(t), len(m),
                          qi.ctypes.data, ti.ctypes.data, ctypes.byref(tp), xyz.ctypes.data, ok.ctypes.data)
    return xyz, ok


def search_pair(cam, Q, T, free_q=None, free_t=None, params=None, t_median_depth=0.0):
    """Matches of one (Q, T) pair as an int32 array (k, 3) of (q_idx, t_idx, dist), sorted
    by q_idx, and the number of descriptor comparisons.  t_median_depth: T's median scene
    depth for the pair-baseline skip (0 = unknown)."""
    p = params or SearchParams()
    keep = []
    q, t = _kf(Q, keep), _kf(T, keep)
    fq, ft = _mask(free_q), _mask(free_t)
    sp = _SearchParams(p.hamming_max, p.ratio_num, p.ratio_den, p.epi_chi2, int(p.epipolar),
                       int(p.resolve), int(p.rot_filter), float(p.epipole_px), int(p.rot_mode),
                       float(p.baseline_min_ratio), float(t_median_depth))
    cap = max(1, min(q.n, t.n) if p.resolve else q.n)
    out = np.zeros((3, cap), np.int32)
    ncmp = ctypes.c_int64(0)
    c = _cam(cam)
    n = lib().orc_search_pair(ctypes.byref(c), ctypes.byref(q), ctypes.byref(t), _ptr(fq),
                              _ptr(ft), ctypes.byref(sp), out[0].ctypes.data,
                              out[1].ctypes.data, out[2].ctypes.data, cap, ctypes.byref(ncmp))
    assert n <= cap
    return np.ascontiguousarray(out[:, :n].T), int(ncmp.value)


def fuse(cam, T, mps, params=None):
    """Fusion candidates of a map-point batch into keyframe T as an int32 array (k, 3) of
    (mp_idx, kp_idx, dist), sorted by mp_idx, and the number of window comparisons."""
    p = params or FuseParams()
    keep = []
    t = _kf(T, keep)
    n = int(mps["n"])
    pos = np.ascontiguousarray(mps["pos"], np.float32)
    nrm = np.ascontiguousarray(mps["normal"], np.float32)
    desc = np.ascontiguousarray(mps["desc"], np.uint8)
    mn = np.ascontiguousarray(mps["min_dist"], np.float32)
    mx = np.ascontiguousarray(mps["max_dist"], np.float32)
    skip = _mask(mps.get("skip"))
    fp = _FuseParams(p.chi2, p.hamming_max, p.radius_scale)
    cap = max(1, n)
    out = np.zeros((3, cap), np.int32)
    ncmp = ctypes.c_int64(0)
    c = _cam(cam)
    k = lib().orc_fuse(ctypes.byref(c), ctypes.byref(t), n, pos.ctypes.data, nrm.ctypes.data,
                       desc.ctypes.data, mn.ctypes.data, mx.ctypes.data, _ptr(skip),
                       ctypes.byref(fp), out[0].ctypes.data, out[1].ctypes.data,
                       out[2].ctypes.data, cap, ctypes.byref(ncmp))
    assert k <= cap
    return np.ascontiguousarray(out[:, :k].T), int(ncmp.value)


def search_step(cam, frames, step, params=None):
    """All pairs of one local-mapping step, in neighbour order: list of match arrays and the
    total number of comparisons."""
    Q = frames[step["q"]]
    res, ncmp = [], 0
    md = step.get("nbr_median_depth")
    for k, f in enumerate(step["nbrs"]):
        ft = None if step.get("nbr_free") is None else step["nbr_free"][k]
        m, c = search_pair(cam, Q, frames[f], step.get("q_free"), ft, params, 0.0 if md is None else float(md[k]))
        res.append(m)
        ncmp += c
    return res, ncmp


def fuse_step(cam, frames, step, params=None):
    if step.get("mps") is None:
        return np.zeros((0, 3), np.int32), 0
    return fuse(cam, frames[step["q"]], step["mps"], params)


def fuse_forward_step(cam, frames, step, params=None):
    """Forward fusion of a step (Sec. IV-D, the other direction): the new keyframe's own map
    points fused into each neighbour in turn, skipping those the neighbour already observes.
    The same per-keyframe fusion as fuse(), applied per neighbour; returns per neighbour an
    int32 (k, 3) array of (mp_idx, kp_idx, dist) and the total number of window comparisons."""
    fw = step.get("fwd_mps")
    if fw is None:
        return [np.zeros((0, 3), np.int32) for _ in step["nbrs"]], 0
    res, ncmp = [], 0
    for k, f in enumerate(step["nbrs"]):
        mps = dict(fw)
        sk = step.get("fwd_skip")
        mps["skip"] = None if sk is None else np.asarray(sk[k], np.uint8)
        r, c = fuse(cam, frames[f], mps, params)
        res.append(r)
        ncmp += c
    return res, ncmp


def culling_redundant(observations, kf, th_obs=3, ratio=0.9):
    """Keyframe culling's redundancy test (Sec. IV-F) by walking observation lists, the
    definition the counter array replaces.  observations: {map point: [(keyframe, level)]};
    kf: the keyframe tested.  A map point of kf, observed by kf at level L, is redundant when at
    least th_obs other keyframes observe it at a level <= L + 1; kf is redundant when more than
    ratio * (its number of map points) are.  Returns (number redundant, redundant)."""
    own = [(m, lv) for m, obs in observations.items() for (k, lv) in obs if k == kf]
    red = 0
    for m, lv in own:
        n = sum(1 for (k, l2) in observations[m] if k != kf and l2 <= lv + 1)
        if n >= th_obs:
            red += 1
    return red, red > ratio * len(own)


class FuseMap:
    """The sequential fuse-apply stage (Sec. IV-D: duplicate pairs are found in parallel and
    merged afterwards, one at a time, keeping the original sequential logic; Sec. II: of two
    duplicate points one is kept and takes over the observations, the other is discarded).
    Plain dictionaries: keyframe -> list (keypoint -> map point or None), map point ->
    {keyframe: keypoint}.

    Readings (the paper gives the stage, not its rule): which point survives follows ORB-SLAM,
    the system the paper restructures: the one with more observations, a tie keeping the point
    being fused; a keyframe that already observes the survivor drops the replaced point's
    keypoint link; a candidate whose point was replaced earlier, or whose target already
    observes it, is skipped."""

    def __init__(self):
        self.kp = {}         # keyframe -> [map point or None] per keypoint
        self.level = {}      # keyframe -> [level] per keypoint
        self.obs = {}        # live map point -> {keyframe: keypoint}
        self.replaced = {}   # replaced map point -> the point that replaced it

    def add_keyframe(self, k, n_kp, level=None):
        assert k not in self.kp
        self.kp[k] = [None] * n_kp
        self.level[k] = [0] * n_kp if level is None else [int(x) for x in level]

    def remove_keyframe(self, k):
        for m in self.kp.pop(k):
            if m is not None:
                del self.obs[m][k]
        del self.level[k]

    def observe(self, k, j, m):
        assert self.kp[k][j] is None and m not in self.replaced and k not in self.obs.get(m, {})
        self.obs.setdefault(m, {})[k] = j
        self.kp[k][j] = m

    def _replace(self, a, b):
        """a is discarded: each of its observations goes to b, unless that keyframe observes b."""
        for k, j in self.obs.pop(a).items():
            if k in self.obs[b]:
                self.kp[k][j] = None
            else:
                self.obs[b][k] = j
                self.kp[k][j] = b
        self.replaced[a] = b

    def fuse(self, k, cands):
        """Applies candidates [(map point, keypoint of k)] in order; returns the counts."""
        st = dict(added=0, merged_into_existing=0, replaced_existing=0, skipped_dead=0, skipped_observed=0)
        for m, j in cands:
            if m in self.replaced:
                st["skipped_dead"] += 1
            elif k in self.obs[m]:
                st["skipped_observed"] += 1
            elif self.kp[k][j] is None:
                self.observe(k, j, m)
                st["added"] += 1
            else:
                p = self.kp[k][j]
                if len(self.obs[p]) > len(self.obs[m]):
                    self._replace(m, p)
                    st["merged_into_existing"] += 1
                else:
                    self._replace(p, m)
                    st["replaced_existing"] += 1
        return st

    def current(self, m):
        """The live point m stands for, following replacements (None if it never existed)."""
        while m in self.replaced:
            m = self.replaced[m]
        return m if m in self.obs else None

    def observations(self):
        """{map point: [(keyframe, level)]} for culling_redundant."""
        return {m: [(k, self.level[k][j]) for k, j in o.items()] for m, o in self.obs.items()}
