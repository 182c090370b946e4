"""GB300-native correspondence search and map-point fusion search for visual-SLAM local
mapping (TurboMap, arXiv 2511.02036, Sec. IV).

Thin Python binding of the C ABI in include/tm.h: every `tm_*` name below is the C function
itself (ctypes), and `Context` / `Plan` / `Server` only marshal numpy arrays or torch tensors
into its structs.  All work runs in the CUDA library libtm.so; importing this package without
it raises.  PyTorch is optional here: tensors are accepted for their device pointers and
`torch.cuda.Stream.cuda_stream` for streams.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib as L
from ._lib import (TM_ERR_BUSY, TM_ERR_CAPACITY, TM_ERR_CUDA, TM_ERR_EXISTS,  # noqa: F401
                   TM_ERR_INVALID_ARG, TM_ERR_NO_MEMORY, TM_ERR_NOT_FOUND, TM_ERR_TIMEOUT,
                   TM_MODE_FUSED, TM_MODE_PER_PAIR, TM_OK, TM_MAX_KP_LIMIT)

_clib = L.load()
for _name in L.SIGNATURES:
    globals()[_name] = getattr(_clib, _name)
LIB_PATH = L.LIB_PATH


class TMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tm status %d: %s" % (status, msg))
        self.status = status


def check(st):
    if st != TM_OK:
        raise TMError(st, _clib.tm_last_error().decode(errors="replace"))
    return st


# --------------------------------------------------------------------------- marshalling

def _ptr(a):
    """Address of a numpy array (host) or torch tensor (host or device); None stays None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _host(a, dtype):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def int_rates(device=0):
    """Measured peak integer-operation rates of a device (tm_measure_int_rates): population
    counts, three-input logic operations and register-resident 256-bit Hamming distances per
    second."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(tm_measure_int_rates(int(device), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))  # noqa: F821
    return dict(popc_per_s=a.value, lop3_per_s=b.value, hamming_per_s=c.value)


def camera_struct(cam):
    return L.tm_camera(int(cam["width"]), int(cam["height"]), float(cam["fx"]), float(cam["fy"]),
                       float(cam["cx"]), float(cam["cy"]))


def keyframe_view(kf, keep):
    """tm_keyframe_view of a dict with desc, xy, angle, level, node (numpy or torch), Tcw."""
    arrs = [_host(kf["desc"], np.uint8), _host(kf["xy"], np.float32), _host(kf["angle"], np.float32),
            _host(kf["level"], np.uint8), _host(kf["node"], np.uint32)]
    keep.extend(arrs)
    v = L.tm_keyframe_view()
    v.n = int(len(arrs[0]))
    v.desc, v.xy, v.angle, v.level, v.node = (_ptr(a) for a in arrs)
    v.Tcw[:] = [float(x) for x in np.asarray(kf["Tcw"], np.float64).reshape(12)]
    return v


def _struct_dtype(ctype):
    """numpy structured dtype with the field offsets and size of a ctypes Structure, so that an
    array of records can be filled column by column and passed as the C array."""
    names, formats, offsets = [], [], []
    for name, ct in ctype._fields_:
        if ct is ctypes.c_void_p:
            fmt = np.uint64
        elif hasattr(ct, "_length_"):
            fmt = (np.dtype(ct._type_), ct._length_)
        else:
            fmt = np.dtype(ct)
        names.append(name)
        formats.append(fmt)
        offsets.append(getattr(ctype, name).offset)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets,
                     "itemsize": ctypes.sizeof(ctype)})


_KF_DT = _struct_dtype(L.tm_keyframe_view)
_STEP_DT = _struct_dtype(L.tm_step)


def keyframe_views(kfs, keep):
    """An array of tm_keyframe_view records (numpy structured, C layout) for keyframe dicts."""
    v = np.zeros(max(1, len(kfs)), _KF_DT)
    for k, kf in enumerate(kfs):
        arrs = [_host(kf["desc"], np.uint8), _host(kf["xy"], np.float32), _host(kf["angle"], np.float32),
                _host(kf["level"], np.uint8), _host(kf["node"], np.uint32)]
        keep.extend(arrs)
        v["n"][k] = len(arrs[0])
        for name, a in zip(("desc", "xy", "angle", "level", "node"), arrs):
            v[name][k] = _ptr(a) or 0
    if len(kfs):
        v["Tcw"][:len(kfs)] = np.asarray([np.asarray(kf["Tcw"], np.float64).reshape(12) for kf in kfs])
    keep.append(v)
    return v


_KF_PACKED = (("desc", np.uint8), ("xy", np.float32), ("angle", np.float32), ("level", np.uint8),
              ("node", np.uint32))
_KF_PACKED_ELT = np.array([32, 8, 4, 1, 4], np.int64)  # bytes per keypoint of each array
_KF_PACKED_COL = [_KF_DT.fields[name][1] // 8 for name, _ in _KF_PACKED]


def keyframe_views_packed(packed, keep):
    """tm_keyframe_view records for keyframes packed one after another in one array per field:
    packed = dict(n=[counts], desc (N, 32), xy (N, 2), angle (N,), level (N,), node (N,),
    Tcw (k, 12) or (k, 3, 4)); numpy arrays or torch tensors (host or device)."""
    n = np.asarray(packed["n"], np.int64).reshape(-1)
    k = len(n)
    v = np.zeros(max(1, k), _KF_DT)
    if not k:
        return v
    start = np.cumsum(n) - n
    # the records as rows of 64-bit words: the five pointer columns in one broadcast, the pose
    # written whole (a few array operations whatever the number of keyframes)
    words = v.view(np.int64).reshape(len(v), _KF_DT.itemsize // 8)
    arrs = [_host(packed[name], dt) for name, dt in _KF_PACKED]
    keep.extend(arrs)
    base = np.array([_ptr(a) or 0 for a in arrs], np.int64)
    cols = base + start[:, None] * _KF_PACKED_ELT
    cols[n == 0] = 0
    words[:, _KF_PACKED_COL] = cols
    t0 = _KF_DT.fields["Tcw"][1] // 8
    words[:, t0:t0 + 12] = np.ascontiguousarray(packed["Tcw"], np.float64).reshape(k, 12).view(np.int64)
    v["n"] = n
    keep.append(v)
    return v


def keyframes_packed(packed, keep):
    """tm_keyframes_packed of keyframes packed one after another (the dict form that
    keyframe_views_packed takes): six pointers and the counts, whatever the number of
    keyframes."""
    n = np.ascontiguousarray(packed["n"], np.int32).reshape(-1)
    tcw = np.ascontiguousarray(packed["Tcw"], np.float64).reshape(len(n), 12)
    arrs = [_host(packed[name], dt) for name, dt in _KF_PACKED]
    keep.extend(arrs + [n, tcw])
    p = L.tm_keyframes_packed()
    p.n, p.Tcw = n.ctypes.data, tcw.ctypes.data
    p.desc, p.xy, p.angle, p.level, p.node = (_ptr(a) for a in arrs)
    keep.append(p)
    return p, n


_MP_FIELDS = (("pos", np.float32, 3), ("normal", np.float32, 3), ("desc", np.uint8, 32),
              ("min_dist", np.float32, 1), ("max_dist", np.float32, 1), ("skip", np.uint8, 1))


def pack_mappoints(mps, pinned=True):
    """The map points of a batch (dict: n, pos, normal, desc, min_dist, max_dist, optional
    skip) copied into one buffer -- page-locked when pinned (torch), else a numpy array --
    each array at a 16-byte aligned offset.  The returned dict holds views into the buffer
    and "block", the buffer: a batch given it uploads its map points with one copy
    (tm_batch_inputs.mps_block) instead of one copy an array."""
    n = int(mps["n"])
    parts = [(f, dt, w) for f, dt, w in _MP_FIELDS if f != "skip" or mps.get("skip") is not None]
    offs, o = {}, 0
    for f, dt, w in parts:
        offs[f] = o
        o = (o + n * w * np.dtype(dt).itemsize + 15) & ~15
    total = max(16, o)
    if pinned:
        import torch
        buf = torch.empty(total, dtype=torch.uint8).pin_memory()
        raw = buf.numpy()
    else:
        buf = raw = np.zeros(total, np.uint8)
    out = dict(n=n, block=buf)
    for f, dt, w in parts:
        x = mps[f]
        a = np.asarray(x.cpu() if hasattr(x, "cpu") else x).astype(dt, copy=False).reshape(n, w) if n else \
            np.zeros((0, w), dt)
        v = raw[offs[f]:offs[f] + a.nbytes].view(dt).reshape((n, w) if w > 1 else (n,))
        v[...] = a.reshape(v.shape)
        out[f] = torch.from_numpy(v) if pinned else v
    return out


def mappoint_view(mps, keep):
    v = L.tm_mappoint_view()
    if mps is None:
        return v
    arrs = [_host(mps["pos"], np.float32), _host(mps["normal"], np.float32), _host(mps["desc"], np.uint8),
            _host(mps["min_dist"], np.float32), _host(mps["max_dist"], np.float32),
            _host(mps.get("skip"), np.uint8)]
    keep.extend(arrs)
    v.n = int(mps["n"])
    v.pos, v.normal, v.desc, v.min_dist, v.max_dist, v.skip = (_ptr(a) for a in arrs)
    return v


@dataclass
class SearchParams:
    hamming_max: int = 50
    ratio_num: int = 3
    ratio_den: int = 5
    epi_chi2: float = 3.84
    epipolar: bool = True
    resolve: bool = True
    rot_filter: bool = True
    mode: int = TM_MODE_FUSED
    lanes_per_query: int = 0
    dense_min: int = 0      # tensor-core blocks for nodes with >= dense_min neighbour keypoints
    epipole_px: float = 0.0  # ORB-family epipole rejection radius at level 0 (0 = off; ORB-SLAM: 10)
    rot_mode: int = 0       # 0: 30 bins of 12 degrees; 1: ORB-family round(rot / 30)
    baseline_min_ratio: float = 0.0  # skip pairs with baseline / median depth below (ORB-SLAM: 0.01)

    @classmethod
    def orb_family(cls, coarse=False, **kw):
        """The ORB-family variants together: epipole rejection at 10 px (scaled by the level),
        rotation bins round(rot / 30), pair-baseline skip below 1 % of the neighbour's median
        depth (the steps must carry that depth).  coarse=True is the family's coarse mode: the
        epipolar-line test is dropped, the epipole rejection kept."""
        kw = dict(dict(epipole_px=10.0, rot_mode=1, baseline_min_ratio=0.01, epipolar=not coarse), **kw)
        return cls(**kw)

    def struct(self):
        return L.tm_search_params(self.hamming_max, self.ratio_num, self.ratio_den, self.epi_chi2,
                                  int(self.epipolar), int(self.resolve), int(self.rot_filter),
                                  int(self.mode), int(self.lanes_per_query), int(self.dense_min),
                                  float(self.epipole_px), int(self.rot_mode), float(self.baseline_min_ratio))


@dataclass
class TriParams:
    """Triangulation of the matches and their acceptance as new map points."""
    cos_parallax_max: float = 0.9998
    chi2: float = 5.991
    ratio_factor: float = 1.5 * 1.2

    def struct(self):
        return L.tm_triangulation_params(self.cos_parallax_max, self.chi2, self.ratio_factor)


@dataclass
class FuseParams:
    chi2: float = 5.99
    hamming_max: int = 50
    radius_scale: float = 3.0

    def struct(self):
        return L.tm_fuse_params(self.chi2, self.hamming_max, self.radius_scale)


@dataclass
class StepTable:
    """Local-mapping steps as columns, for batches whose masks and map points are already
    packed (tm_step fields, one entry per step; the neighbour ids of all steps back to back in
    step order): kf_id, n_nbrs, nbr_ids, and optionally q_free_off / nbr_free_off (byte offsets
    into the batch's masks, -1 = all free) and mp_begin / mp_count (range of the batch's map
    points).  batch_run and plan take it in place of a list of step dicts and then need no
    Python loop over the pairs."""
    kf_id: np.ndarray
    n_nbrs: np.ndarray
    nbr_ids: np.ndarray
    q_free_off: np.ndarray = None
    nbr_free_off: np.ndarray = None
    mp_begin: np.ndarray = None
    mp_count: np.ndarray = None
    fwd_mp_begin: np.ndarray = None
    fwd_mp_count: np.ndarray = None
    fwd_skip_off: np.ndarray = None
    nbr_median_depth: np.ndarray = None  # per neighbour, aligned with nbr_ids (float32)

    @classmethod
    def from_steps(cls, steps):
        """From step dicts with kf_id, nbrs and the optional offset fields above."""
        n = len(steps)
        cnt = np.fromiter((len(s["nbrs"]) for s in steps), np.int32, n)
        col = lambda k, d, dt: np.fromiter((s.get(k, d) for s in steps), dt, n)  # noqa: E731
        return cls(np.fromiter((s["kf_id"] for s in steps), np.uint64, n), cnt,
                   np.fromiter((t for s in steps for t in s["nbrs"]), np.uint64, int(cnt.sum())),
                   col("q_free_off", -1, np.int64), col("nbr_free_off", -1, np.int64),
                   col("mp_begin", 0, np.int32), col("mp_count", 0, np.int32),
                   col("fwd_mp_begin", 0, np.int32), col("fwd_mp_count", 0, np.int32),
                   col("fwd_skip_off", -1, np.int64))

    def __len__(self):
        return len(self.kf_id)

    def _cached(self, name, make):
        v = self.__dict__.get(name)
        if v is None:
            v = make()
            self.__dict__[name] = v
        return v

    def n_pairs(self):
        """Neighbour pairs of all steps (read at first use, like the records)."""
        return self._cached("_n_pairs", lambda: int(np.sum(np.asarray(self.n_nbrs, np.int64))))

    def lists(self):
        """(kf ids, neighbour counts) as Python lists (read at first use)."""
        return self._cached("_lists", lambda: (np.asarray(self.kf_id, np.uint64).tolist(),
                                                 np.asarray(self.n_nbrs, np.int64).tolist()))

    def records(self, keep):
        """tm_step records (numpy structured array, C layout); the arrays they point into are
        appended to keep.  Built at the table's first use and kept with it: a table is read
        once, so build a new one for new steps rather than changing its columns in place."""
        cached = self.__dict__.get("_records")
        if cached is not None:
            keep.extend(cached)
            return cached[-1]
        mark = len(keep)
        arr = self._build_records(keep)
        self.__dict__["_records"] = list(keep[mark:])
        return arr

    def _build_records(self, keep):
        n = len(self.kf_id)
        arr = np.zeros(max(1, n), _STEP_DT)
        cnt = np.asarray(self.n_nbrs, np.int64)
        nbrs = np.ascontiguousarray(self.nbr_ids, np.uint64)
        keep.append(nbrs)
        off = np.concatenate([[0], np.cumsum(cnt)[:-1]]) if n else np.zeros(0, np.int64)
        arr["kf_id"][:n] = self.kf_id
        arr["n_nbrs"][:n] = cnt
        arr["nbr_ids"][:n] = np.where(cnt > 0, nbrs.ctypes.data + 8 * off, 0)
        arr["q_free_off"][:n] = -1 if self.q_free_off is None else self.q_free_off
        arr["nbr_free_off"][:n] = -1 if self.nbr_free_off is None else self.nbr_free_off
        arr["mp_begin"][:n] = 0 if self.mp_begin is None else self.mp_begin
        arr["mp_count"][:n] = 0 if self.mp_count is None else self.mp_count
        arr["fwd_mp_begin"][:n] = 0 if self.fwd_mp_begin is None else self.fwd_mp_begin
        arr["fwd_mp_count"][:n] = 0 if self.fwd_mp_count is None else self.fwd_mp_count
        arr["fwd_skip_off"][:n] = -1 if self.fwd_skip_off is None else self.fwd_skip_off
        if self.nbr_median_depth is not None:
            md = np.ascontiguousarray(self.nbr_median_depth, np.float32)
            assert len(md) == len(nbrs)
            keep.append(md)
            arr["nbr_median_depth"][:n] = np.where(cnt > 0, md.ctypes.data + 4 * off, 0)
        keep.append(arr)
        return arr


def _split(arr, offsets):
    return [arr[offsets[k]:offsets[k + 1]] for k in range(len(offsets) - 1)]


def pack_batch(steps, kf_sizes):
    """Concatenate the masks and map points of local-mapping steps into one batch.

    steps: dicts with kf_id, nbrs (ids), optional q_free [n_Q], nbr_free (list of [n_T]),
    optional mps (map-point dict, fused into kf_id), optional fwd_mps (the new keyframe's own
    map points, fused into every neighbour) with fwd_skip (per neighbour a [fwd n] uint8
    array, 1 = already observed by that neighbour).  kf_sizes: kf_id -> keypoint count.
    Returns (tm_step array, masks uint8, concatenated map points dict, keep-alive list)."""
    st = (L.tm_step * max(1, len(steps)))()
    masks, keep = [], []
    cols = {k: [] for k in ("pos", "normal", "desc", "min_dist", "max_dist", "skip")}
    moff = mo = 0
    any_skip = False
    for k, s in enumerate(steps):
        nb = np.ascontiguousarray(s["nbrs"], np.uint64)
        keep.append(nb)
        st[k].kf_id = int(s["kf_id"])
        st[k].nbr_ids = nb.ctypes.data if len(nb) else None
        st[k].n_nbrs = len(nb)
        st[k].q_free_off = -1
        st[k].nbr_free_off = -1
        st[k].fwd_skip_off = -1
        if s.get("nbr_median_depth") is not None:
            md = np.ascontiguousarray(s["nbr_median_depth"], np.float32)
            assert len(md) == len(nb)
            keep.append(md)
            st[k].nbr_median_depth = md.ctypes.data
        if s.get("q_free") is not None:
            st[k].q_free_off = moff
            masks.append(np.asarray(s["q_free"], np.uint8))
            moff += len(masks[-1])
        if s.get("nbr_free") is not None:
            st[k].nbr_free_off = moff
            for m in s["nbr_free"]:
                masks.append(np.asarray(m, np.uint8))
                moff += len(masks[-1])
        mp = s.get("mps")
        st[k].mp_begin = mo
        st[k].mp_count = 0 if mp is None else int(mp["n"])
        if mp is not None and mp["n"]:
            for c in cols:
                if c == "skip":
                    sk = mp.get("skip")
                    any_skip |= sk is not None
                    cols[c].append(np.zeros(mp["n"], np.uint8) if sk is None else np.asarray(sk, np.uint8))
                else:
                    cols[c].append(np.asarray(mp[c]))
            mo += int(mp["n"])
        fw = s.get("fwd_mps")
        st[k].fwd_mp_begin = mo
        st[k].fwd_mp_count = 0 if fw is None else int(fw["n"])
        if fw is not None and fw["n"]:
            for c in cols:  # (their per-batch skip bytes are unused: forward items skip by fwd_skip)
                cols[c].append(np.zeros(fw["n"], np.uint8) if c == "skip" else np.asarray(fw[c]))
            mo += int(fw["n"])
            if s.get("fwd_skip") is not None:
                st[k].fwd_skip_off = moff
                for m in s["fwd_skip"]:
                    masks.append(np.asarray(m, np.uint8))
                    moff += len(masks[-1])
    mask_arr = np.ascontiguousarray(np.concatenate(masks) if masks else np.zeros(0, np.uint8))
    mps = dict(n=mo,
               pos=np.ascontiguousarray(np.concatenate(cols["pos"]) if mo else np.zeros((0, 3)), np.float32),
               normal=np.ascontiguousarray(np.concatenate(cols["normal"]) if mo else np.zeros((0, 3)), np.float32),
               desc=np.ascontiguousarray(np.concatenate(cols["desc"]) if mo else np.zeros((0, 32)), np.uint8),
               min_dist=np.ascontiguousarray(np.concatenate(cols["min_dist"]) if mo else np.zeros(0), np.float32),
               max_dist=np.ascontiguousarray(np.concatenate(cols["max_dist"]) if mo else np.zeros(0), np.float32),
               skip=np.ascontiguousarray(np.concatenate(cols["skip"]), np.uint8) if (mo and any_skip) else None)
    return st, mask_arr, mps, keep


class BatchResult:
    """Results of a batch: per pair (in step then neighbour order) an int32 (k, 3) array of
    (q_idx, t_idx, dist); per step an int32 (k, 3) array of (mp_idx, kp_idx, dist); per pair
    the forward-fusion candidates (the step's new keyframe's map points, mp_idx relative to
    fwd_mp_begin, in the neighbour's keypoints)."""

    def __init__(self, matches, pair_offsets, fuse, fuse_offsets, ncmp_search, ncmp_fuse,
                 fwd=None, fwd_offsets=None, ncmp_fwd=0, points=None, point_ok=None):
        self.matches = matches
        self.pair_offsets = pair_offsets
        self.fuse = fuse
        self.fuse_offsets = fuse_offsets
        self.fwd = np.zeros((0, 3), np.int32) if fwd is None else fwd
        self.fwd_offsets = np.zeros(len(pair_offsets), np.int32) if fwd_offsets is None else fwd_offsets
        self._pairs = self._fuses = self._fwds = None
        self.n_comparisons_search = ncmp_search
        self.n_comparisons_fuse = ncmp_fuse
        self.n_comparisons_fwd = ncmp_fwd
        self.points = points        # (n_matches, 3) float32 with triangulation, else None
        self.point_ok = point_ok    # (n_matches,) uint8: accepted as a new map point

    @property
    def fwds(self):
        """Per pair, its forward-fusion rows of `fwd` (views, split on first use)."""
        if self._fwds is None:
            self._fwds = _split(self.fwd, self.fwd_offsets)
        return self._fwds

    @property
    def pairs(self):
        """Per pair, its rows of `matches` (views, split on first use)."""
        if self._pairs is None:
            self._pairs = _split(self.matches, self.pair_offsets)
        return self._pairs

    @property
    def fuses(self):
        """Per step, its rows of `fuse` (views, split on first use)."""
        if self._fuses is None:
            self._fuses = _split(self.fuse, self.fuse_offsets)
        return self._fuses


def _result_struct(match_cap, n_pairs, fuse_cap, n_steps, fwd_cap=0, tri=False):
    m = np.zeros((max(1, match_cap), 3), np.int32)
    po = np.zeros(n_pairs + 1, np.int32)
    f = np.zeros((max(1, fuse_cap), 3), np.int32)
    fo = np.zeros(n_steps + 1, np.int32)
    w = np.zeros((max(1, fwd_cap), 3), np.int32)
    wo = np.zeros(n_pairs + 1, np.int32)
    r = L.tm_batch_result()
    r.matches, r.match_cap, r.pair_offsets = m.ctypes.data, match_cap, po.ctypes.data
    r.fuse, r.fuse_cap, r.fuse_offsets = f.ctypes.data, fuse_cap, fo.ctypes.data
    r.fwd, r.fwd_cap, r.fwd_offsets = w.ctypes.data, fwd_cap, wo.ctypes.data
    pt = ok = None
    if tri:
        pt = np.zeros((max(1, match_cap), 3), np.float32)
        ok = np.zeros(max(1, match_cap), np.uint8)
        r.points, r.point_ok = pt.ctypes.data, ok.ctypes.data
    return r, (m, po, f, fo, w, wo, pt, ok)


def _collect(r, bufs, copy=True):
    m, po, f, fo, w, wo, pt, ok = bufs
    n = r.n_matches
    c = (lambda a: a.copy()) if copy else (lambda a: a)
    return BatchResult(c(m[:n]), c(po), c(f[:r.n_fuse]), c(fo),
                       int(r.n_comparisons_search), int(r.n_comparisons_fuse),
                       c(w[:r.n_fwd]), c(wo), int(r.n_comparisons_fwd),
                       None if pt is None else c(pt[:n]), None if ok is None else c(ok[:n]))


def _fwd_cap(steps):
    """Forward-fusion output capacity: every neighbour of a step times its forward map points."""
    if isinstance(steps, StepTable):
        if steps.fwd_mp_count is None:
            return 0
        return steps._cached("_fwd_cap", lambda: int((np.asarray(steps.fwd_mp_count, np.int64) *
                                                      np.asarray(steps.n_nbrs, np.int64)).sum()))
    tot = 0
    for s in steps:
        c = s.get("fwd_mp_count")
        if c is None:
            fw = s.get("fwd_mps")
            c = 0 if fw is None else int(fw["n"])
        tot += int(c) * len(s["nbrs"])
    return tot


def _result_caps(steps, kf_sizes, resolve=True, default=TM_MAX_KP_LIMIT):
    """Output capacities from the known keyframe sizes (unknown ids: the C call reports them)."""
    g = kf_sizes.get
    if isinstance(steps, StepTable):
        # per step only: at most n_Q matches per pair (the looser bound; no lookup per pair)
        kf, nn = steps.lists()
        mc = sum(g(k, default) * n for k, n in zip(kf, nn))
        fc = steps._cached("_mp_total", lambda: 0 if steps.mp_count is None else
                           int(np.asarray(steps.mp_count, np.int64).sum()))
        return mc, fc
    nq = np.fromiter((g(int(s["kf_id"]), default) for s in steps), np.int64, len(steps))
    cnt = np.fromiter((len(s["nbrs"]) for s in steps), np.int64, len(steps))
    nt = np.fromiter((g(int(t), default) for s in steps for t in s["nbrs"]), np.int64, int(cnt.sum()))
    nqp = np.repeat(nq, cnt)
    mc = int(np.minimum(nqp, nt).sum() if resolve else nqp.sum())
    fc = sum(int(s["mps"]["n"]) for s in steps if s.get("mps") is not None)
    return mc, fc


class ResultBuffers:
    """Host result buffers (pinned when torch is available, so that the results come back by
    DMA), grown as needed.  A context keeps one set for its one-shot calls and copies the
    results out of it; a caller may own sets of its own instead and pass one as `out` to
    Context.batch_run / batch_finish: the BatchResult's arrays are then views into that set,
    with no copy, valid until the set is passed to another call (one set per batch in flight)."""

    def __init__(self):
        self.m = self.po = self.f = self.fo = self.w = self.wo = self.pt = self.ok = None
        self._last = None  # (capacities, result struct, views) of the previous call

    @staticmethod
    def _grow(a, n, width):
        if a is not None and a.shape[0] >= n:
            return a
        n = max(n, 1024)
        try:
            import torch
            t = torch.empty((n, width) if width else (n,), dtype=torch.int32).pin_memory()
            return t.numpy()
        except Exception:  # no torch or no CUDA runtime: pageable memory
            return np.empty((n, width) if width else (n,), np.int32)

    def struct(self, match_cap, n_pairs, fuse_cap, n_steps, fwd_cap=0, tri=False):
        key = (match_cap, n_pairs, fuse_cap, n_steps, fwd_cap, tri)
        if self._last is not None and self._last[0] == key:
            return self._last[1], self._last[2]
        self.m = self._grow(self.m, max(1, match_cap), 3)
        self.po = self._grow(self.po, n_pairs + 1, 0)
        self.f = self._grow(self.f, max(1, fuse_cap), 3)
        self.fo = self._grow(self.fo, n_steps + 1, 0)
        self.w = self._grow(self.w, max(1, fwd_cap), 3)
        self.wo = self._grow(self.wo, n_pairs + 1, 0)
        r = L.tm_batch_result()
        r.matches, r.match_cap, r.pair_offsets = self.m.ctypes.data, match_cap, self.po.ctypes.data
        r.fuse, r.fuse_cap, r.fuse_offsets = self.f.ctypes.data, fuse_cap, self.fo.ctypes.data
        r.fwd, r.fwd_cap, r.fwd_offsets = self.w.ctypes.data, fwd_cap, self.wo.ctypes.data
        pt = ok = None
        if tri:
            self.pt = self._grow_f(self.pt, max(1, match_cap))
            self.ok = self._grow_u8(self.ok, max(1, match_cap))
            pt, ok = self.pt, self.ok
            r.points, r.point_ok = pt.ctypes.data, ok.ctypes.data
        bufs = (self.m, self.po[:n_pairs + 1], self.f, self.fo[:n_steps + 1], self.w, self.wo[:n_pairs + 1], pt, ok)
        self._last = (key, r, bufs)
        return r, bufs

    @staticmethod
    def _grow_f(a, n):
        return a if a is not None and a.shape[0] >= n else np.empty((max(n, 1024), 3), np.float32)

    @staticmethod
    def _grow_u8(a, n):
        return a if a is not None and a.shape[0] >= n else np.empty(max(n, 1024), np.uint8)


class ObsCounter:
    """Keyframe-culling observation counters (tm_obs_*, host-side): per map point the number of
    keyframe observations at each pyramid level."""

    def __init__(self, max_mps):
        h = ctypes.c_void_p()
        check(tm_obs_create(int(max_mps), ctypes.byref(h)))  # noqa: F821
        self.handle = h

    @staticmethod
    def _arrays(mp, level):
        mp = np.ascontiguousarray(mp, np.int32)
        level = np.ascontiguousarray(level, np.uint8)
        assert mp.shape == level.shape
        return mp, level

    def add(self, mp, level):
        mp, level = self._arrays(mp, level)
        check(tm_obs_add(self.handle, len(mp), mp.ctypes.data, level.ctypes.data))  # noqa: F821

    def remove(self, mp, level):
        mp, level = self._arrays(mp, level)
        check(tm_obs_remove(self.handle, len(mp), mp.ctypes.data, level.ctypes.data))  # noqa: F821

    def redundant(self, mp, level, th_obs=3, ratio=0.9):
        """(number of redundant map points, keyframe redundant) for a keyframe's observations."""
        mp, level = self._arrays(mp, level)
        nr, red = ctypes.c_int32(), ctypes.c_int32()
        check(tm_obs_redundant(self.handle, len(mp), mp.ctypes.data, level.ctypes.data,  # noqa: F821
                               int(th_obs), float(ratio), ctypes.byref(nr), ctypes.byref(red)))
        return nr.value, bool(red.value)

    def close(self):
        if self.handle:
            check(tm_obs_destroy(self.handle))  # noqa: F821
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Map:
    """The host-side map of the fuse-apply stage (tm_map_*): per keyframe a keypoint -> map point
    table and keypoint levels, per map point its observations, and the culling counters.  The
    fusion search (GPU) lists candidates; fuse_apply merges them in order (Sec. IV-D)."""

    def __init__(self, max_mps):
        h = ctypes.c_void_p()
        check(tm_map_create(int(max_mps), ctypes.byref(h)))  # noqa: F821
        self.handle = h

    def add_keyframe(self, kf_id, n_kp, level=None):
        lv = None if level is None else np.ascontiguousarray(level, np.uint8)
        assert lv is None or len(lv) == n_kp
        check(tm_map_add_keyframe(self.handle, int(kf_id), int(n_kp), _ptr(lv)))  # noqa: F821

    def remove_keyframe(self, kf_id):
        check(tm_map_remove_keyframe(self.handle, int(kf_id)))  # noqa: F821

    def add_observations(self, kf_id, kp, mp):
        kp = np.ascontiguousarray(kp, np.int32)
        mp = np.ascontiguousarray(mp, np.int32)
        assert kp.shape == mp.shape
        check(tm_map_add_observations(self.handle, int(kf_id), len(kp), kp.ctypes.data,  # noqa: F821
                                      mp.ctypes.data))

    def fuse_apply(self, kf_id, cands, mp_ids=None):
        """cands: int32 (k, 3) (mp_idx, kp_idx, dist) rows as tm_fuse / batch results give them;
        mp_ids: the batch's map point ids (None: mp_idx is the id).  Returns the call's counts."""
        c = np.ascontiguousarray(np.asarray(cands, np.int32).reshape(-1, 3))
        ids = None if mp_ids is None else np.ascontiguousarray(mp_ids, np.int32)
        st = L.tm_fuse_apply_stats()
        check(tm_map_fuse_apply(self.handle, int(kf_id), len(c), c.ctypes.data if len(c) else None,  # noqa: F821
                                _ptr(ids), 0 if ids is None else len(ids), ctypes.byref(st)))
        return {f: int(getattr(st, f)) for f, _ in L.tm_fuse_apply_stats._fields_}

    def keyframe_points(self, kf_id, n_kp):
        out = np.zeros(max(1, n_kp), np.int32)
        check(tm_map_keyframe_points(self.handle, int(kf_id), int(n_kp), out.ctypes.data))  # noqa: F821
        return out[:n_kp]

    def point_info(self, mps):
        """(live, current, n_obs) per map point: live 1 / 0 replaced / -1 never existed."""
        mp = np.ascontiguousarray(mps, np.int32)
        n = len(mp)
        live, cur, nobs = (np.zeros(max(1, n), np.int32) for _ in range(3))
        check(tm_map_point_info(self.handle, n, mp.ctypes.data, live.ctypes.data, cur.ctypes.data,  # noqa: F821
                                nobs.ctypes.data))
        return live[:n], cur[:n], nobs[:n]

    def redundant(self, kf_id, th_obs=3, ratio=0.9):
        nr, red = ctypes.c_int32(), ctypes.c_int32()
        check(tm_map_redundant(self.handle, int(kf_id), int(th_obs), float(ratio),  # noqa: F821
                               ctypes.byref(nr), ctypes.byref(red)))
        return nr.value, bool(red.value)

    def close(self):
        if self.handle:
            check(tm_map_destroy(self.handle))  # noqa: F821
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Context:
    """A tm_ctx: one GPU, one camera, a keyframe store of max_kp-keypoint slots."""

    def __init__(self, cam, max_kp=4096, budget=0, device=0):
        self.cam = dict(cam)
        self.max_kp = max_kp
        h = ctypes.c_void_p()
        c = camera_struct(cam)
        check(tm_ctx_create(device, ctypes.byref(c), max_kp, budget, ctypes.byref(h)))  # noqa: F821
        self.handle = h
        self.sizes = {}
        self._res = None

    def close(self):
        if self.handle:
            check(tm_ctx_destroy(self.handle))  # noqa: F821
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- store
    def add_keyframe(self, kf_id, kf, stream=None):
        keep = []
        v = keyframe_view(kf, keep)
        check(tm_store_add_keyframe(self.handle, int(kf_id), ctypes.byref(v), _stream(stream)))  # noqa: F821
        self.sizes[int(kf_id)] = v.n

    def add_keyframes(self, ids, kfs, stream=None):
        keep = []
        n = len(ids)
        views = (L.tm_keyframe_view * max(1, n))()
        for k, kf in enumerate(kfs):
            views[k] = keyframe_view(kf, keep)
        idarr = np.ascontiguousarray(ids, np.uint64)
        check(tm_store_add_keyframes(self.handle, n, idarr.ctypes.data, views, _stream(stream)))  # noqa: F821
        for k in range(n):
            self.sizes[int(ids[k])] = views[k].n

    def remove_keyframe(self, kf_id):
        check(tm_store_remove_keyframe(self.handle, int(kf_id)))  # noqa: F821
        self.sizes.pop(int(kf_id), None)

    def remove_keyframes(self, kf_ids):
        """Removes several keyframes in one call (all or nothing)."""
        ids = np.ascontiguousarray(kf_ids, np.uint64)
        check(tm_store_remove_keyframes(self.handle, len(ids), ids.ctypes.data))  # noqa: F821
        for i in ids.tolist():
            self.sizes.pop(i, None)

    def reserve(self, n_slots):
        """Allocates keyframe slots ahead (tm_store_reserve): later additions allocate nothing."""
        check(tm_store_reserve(self.handle, int(n_slots)))  # noqa: F821

    def keyframe_size(self, kf_id):
        n = ctypes.c_int32()
        check(tm_store_keyframe_size(self.handle, int(kf_id), ctypes.byref(n)))  # noqa: F821
        return n.value

    def stats(self):
        s = L.tm_store_stats()
        check(tm_store_get_stats(self.handle, ctypes.byref(s)))  # noqa: F821
        return {f: getattr(s, f) for f, _ in s._fields_}

    # ---------------------------------------------------------------- search / fuse
    def search(self, kf_id, nbrs, q_free=None, nbr_free=None, params=None, stream=None):
        """Per-pair match arrays (q_idx, t_idx, dist) in neighbour order, and the number of
        descriptor comparisons."""
        p = (params or SearchParams()).struct()
        nb = np.ascontiguousarray(nbrs, np.uint64)
        # result capacity from the known sizes; unknown ids are reported by the C call
        nq = self.sizes.get(int(kf_id), self.max_kp)
        cap = sum(min(nq, self.sizes.get(int(t), self.max_kp)) if p.resolve else nq for t in nb)
        out = np.zeros((max(1, cap), 3), np.int32)
        po = np.zeros(len(nb) + 1, np.int32)
        n_out, ncmp = ctypes.c_size_t(), ctypes.c_uint64()
        qf = _host(q_free, np.uint8)
        if nbr_free is not None and isinstance(nbr_free, (list, tuple)):
            nbr_free = np.concatenate([np.asarray(m, np.uint8) for m in nbr_free]) if len(nbr_free) else None
        nf = _host(nbr_free, np.uint8)
        check(tm_search_triangulation(self.handle, int(kf_id), nb.ctypes.data if len(nb) else None,  # noqa: F821
                                      len(nb), ctypes.byref(p), _ptr(qf), _ptr(nf), out.ctypes.data,
                                      cap, ctypes.byref(n_out), po.ctypes.data, ctypes.byref(ncmp),
                                      _stream(stream)))
        return _split(out[:n_out.value].copy(), po), int(ncmp.value)

    def fuse(self, kf_id, mps, params=None, stream=None):
        p = (params or FuseParams()).struct()
        keep = []
        v = mappoint_view(mps, keep)
        out = np.zeros((max(1, v.n), 3), np.int32)
        n_out, ncmp = ctypes.c_size_t(), ctypes.c_uint64()
        check(tm_fuse(self.handle, int(kf_id), ctypes.byref(v), ctypes.byref(p), out.ctypes.data,  # noqa: F821
                      v.n, ctypes.byref(n_out), ctypes.byref(ncmp), _stream(stream)))
        return out[:n_out.value].copy(), int(ncmp.value)

    # ---------------------------------------------------------------- batches
    def _inputs(self, steps, masks=None, mps=None, new=None):
        keep = []
        if masks is None and mps is None:
            st, masks, mps, k2 = pack_batch(steps, self.sizes)
            keep.extend(k2)
        elif isinstance(steps, StepTable):
            arr = steps.records(keep)
            st = arr.ctypes.data
        else:
            n = len(steps)
            arr = np.zeros(max(1, n), _STEP_DT)
            cnt = np.fromiter((len(s["nbrs"]) for s in steps), np.int64, n)
            nbrs = np.fromiter((t for s in steps for t in s["nbrs"]), np.uint64, int(cnt.sum()))
            keep.append(nbrs)
            off = np.concatenate([[0], np.cumsum(cnt)[:-1]]) if n else np.zeros(0, np.int64)
            arr["kf_id"][:n] = np.fromiter((s["kf_id"] for s in steps), np.uint64, n)
            arr["n_nbrs"][:n] = cnt
            arr["nbr_ids"][:n] = np.where(cnt > 0, nbrs.ctypes.data + 8 * off, 0)
            arr["q_free_off"][:n] = np.fromiter((s.get("q_free_off", -1) for s in steps), np.int64, n)
            arr["nbr_free_off"][:n] = np.fromiter((s.get("nbr_free_off", -1) for s in steps), np.int64, n)
            arr["mp_begin"][:n] = np.fromiter((s.get("mp_begin", 0) for s in steps), np.int64, n)
            arr["mp_count"][:n] = np.fromiter((s.get("mp_count", 0) for s in steps), np.int64, n)
            arr["fwd_mp_begin"][:n] = np.fromiter((s.get("fwd_mp_begin", 0) for s in steps), np.int64, n)
            arr["fwd_mp_count"][:n] = np.fromiter((s.get("fwd_mp_count", 0) for s in steps), np.int64, n)
            arr["fwd_skip_off"][:n] = np.fromiter((s.get("fwd_skip_off", -1) for s in steps), np.int64, n)
            mds = [None if s.get("nbr_median_depth") is None else np.ascontiguousarray(s["nbr_median_depth"], np.float32)
                   for s in steps]
            keep.extend(m for m in mds if m is not None)
            arr["nbr_median_depth"][:n] = [0 if m is None else m.ctypes.data for m in mds]
            st = arr.ctypes.data
            keep.append(arr)
        inp = L.tm_batch_inputs()
        keep.append(masks)
        inp.masks = _ptr(masks) if masks is not None and len(masks) else None
        inp.mask_bytes = 0 if masks is None else int(np.prod(masks.shape)) if isinstance(masks, np.ndarray) else masks.numel()
        inp.mps = mappoint_view(mps if mps is not None and mps["n"] else None, keep)
        blk = mps.get("block") if isinstance(mps, dict) and mps["n"] else None
        if blk is not None:
            # one allocation holding every array (pack_mappoints): uploaded with one copy
            keep.append(blk)
            inp.mps_block = _ptr(blk)
            inp.mps_block_bytes = int(blk.nbytes) if isinstance(blk, np.ndarray) else blk.numel() * blk.element_size()
        if new is not None:
            ids, kfs = new
            idarr = np.ascontiguousarray(ids, np.uint64)
            keep.append(idarr)
            inp.n_new, inp.new_ids = len(idarr), idarr.ctypes.data
            if isinstance(kfs, dict):
                # packed keyframes: one record of six arrays (tm_keyframes_packed)
                pk, counts = keyframes_packed(kfs, keep)
                assert len(counts) == len(idarr)
                inp.new_packed = ctypes.addressof(pk)
            else:
                views = keyframe_views(kfs, keep)
                counts = views["n"][:len(idarr)]
                inp.new_kfs = views.ctypes.data
            self.sizes.update(zip(idarr.tolist(), counts.tolist()))
        keep.append(st)
        return st, inp, keep

    def batch_run(self, steps, masks=None, mps=None, sp=None, fp=None, stream=None, new=None, tri=None,
                  out=None):
        """One-shot batch (tm_batch_run).  Without masks/mps the steps carry their own
        q_free / nbr_free / mps and are packed here.  new = (ids, keyframes) entering the
        store with the batch: a list of keyframe dicts, or one packed dict (see
        keyframe_views_packed).  tri = TriParams(): triangulate every match (res.points,
        res.point_ok).  out = a caller's ResultBuffers: the results as views into it."""
        sp = sp or SearchParams()
        st, inp, keep = self._inputs(steps, masks, mps, new)
        if tri is not None:
            ts = tri.struct()
            keep.append(ts)
            inp.tri = ctypes.addressof(ts)
        mc, fc = _result_caps(steps, self.sizes, sp.resolve)
        if masks is not None or mps is not None:
            fc = max(fc, int(mps["n"]) if mps is not None else 0)
        if self._res is None:
            self._res = ResultBuffers()
        n_pairs = steps.n_pairs() if isinstance(steps, StepTable) else sum(len(s["nbrs"]) for s in steps)
        r, bufs = (out or self._res).struct(mc, n_pairs, fc, len(steps), _fwd_cap(steps), tri is not None)
        sps, fps = sp.struct(), (fp or FuseParams()).struct()
        try:
            check(tm_batch_run(self.handle, st, len(steps), ctypes.byref(inp), ctypes.byref(sps),  # noqa: F821
                               ctypes.byref(fps), ctypes.byref(r), _stream(stream)))
        except TMError:
            if new is not None:
                for i in new[0]:
                    self.sizes.pop(int(i), None)
            raise
        return _collect(r, bufs, copy=out is None)

    def batch_begin(self, steps, masks=None, mps=None, sp=None, fp=None, new=None, tri=None):
        """Asynchronous batch_run (tm_batch_begin): enqueues the batch and returns a ticket for
        batch_finish.  The input arrays must stay alive and unchanged until then (the context
        keeps references to them); at most L.TM_BATCH_INFLIGHT batches are in flight."""
        sp = sp or SearchParams()
        st, inp, keep = self._inputs(steps, masks, mps, new)
        if tri is not None:
            ts = tri.struct()
            keep.append(ts)
            inp.tri = ctypes.addressof(ts)
        mc, fc = _result_caps(steps, self.sizes, sp.resolve)
        if masks is not None or mps is not None:
            fc = max(fc, int(mps["n"]) if mps is not None else 0)
        n_pairs = steps.n_pairs() if isinstance(steps, StepTable) else sum(len(s["nbrs"]) for s in steps)
        sps, fps = sp.struct(), (fp or FuseParams()).struct()
        keep.extend([sps, fps])
        t = ctypes.c_uint64()
        try:
            check(tm_batch_begin(self.handle, st, len(steps), ctypes.byref(inp), ctypes.byref(sps),  # noqa: F821
                                 ctypes.byref(fps), ctypes.byref(t)))
        except TMError:
            if new is not None:
                for i in new[0]:
                    self.sizes.pop(int(i), None)
            raise
        if not hasattr(self, "_inflight"):
            self._inflight = {}
        self._inflight[t.value] = (keep, (mc, n_pairs, fc, len(steps), _fwd_cap(steps), tri is not None),
                                   None if new is None else list(new[0]))
        return t.value

    def batch_finish(self, ticket, out=None):
        """Waits for a batch begun by batch_begin and returns its BatchResult (with out = a
        caller's ResultBuffers: views into it).  The wait does not hold the context: another
        thread may begin batches meanwhile (finishes on several threads at once need out=)."""
        keep, caps, new_ids = self._inflight.pop(ticket)
        if self._res is None:
            self._res = ResultBuffers()
        r, bufs = (out or self._res).struct(*caps)
        try:
            check(tm_batch_finish(self.handle, ticket, ctypes.byref(r)))  # noqa: F821
        except TMError:
            for i in new_ids or []:
                self.sizes.pop(int(i), None)
            raise
        return _collect(r, bufs, copy=out is None)

    def last_host_times(self):
        """Host microseconds of the phases of the last batch_run (tm_batch_last_host_times):
        dict(prepare, launch, wait, download)."""
        us = np.zeros(4, np.float64)
        check(tm_batch_last_host_times(self.handle, us.ctypes.data))  # noqa: F821
        return dict(zip(("prepare", "launch", "wait", "download"), us.tolist()))

    def debug_set(self, what, value):
        """Test hooks of the context (tm_debug_set): L.TM_DEBUG_WAIT_LIMIT (SM cycles),
        L.TM_DEBUG_STARVE_WAITS (bounded device waits run out), and launch choices otherwise
        left to the autotuner (L.TM_DEBUG_QUERIES_PER_LANE, L.TM_DEBUG_PERSISTENT,
        L.TM_DEBUG_L2_PREFETCH, L.TM_DEBUG_BRANCH_PRIORITY)."""
        check(tm_debug_set(self.handle, int(what), int(value)))  # noqa: F821

    def plan(self, steps, masks=None, mps=None, sp=None, fp=None, new=None, tri=None):
        return Plan(self, steps, masks, mps, sp or SearchParams(), fp or FuseParams(), new, tri)

    def server(self, **cfg):
        return Server(self, **cfg)


class Plan:
    """A prepared batch (tm_plan): inputs resident on the GPU, launch captured in a graph."""

    def __init__(self, ctx, steps, masks, mps, sp, fp, new=None, tri=None):
        self.ctx = ctx
        st, inp, self._keep = ctx._inputs(steps, masks, mps, new)
        self.tri = tri is not None
        if tri is not None:
            ts = tri.struct()
            self._keep.append(ts)
            inp.tri = ctypes.addressof(ts)
        self.caps = _result_caps(steps, ctx.sizes, sp.resolve)
        if mps is not None:
            self.caps = (self.caps[0], max(self.caps[1], int(mps["n"])))
        self.n_pairs = int(np.sum(steps.n_nbrs)) if isinstance(steps, StepTable) else sum(len(s["nbrs"]) for s in steps)
        self.n_steps = len(steps)
        self.fwd_cap = _fwd_cap(steps)
        h = ctypes.c_void_p()
        sps, fps = sp.struct(), fp.struct()
        check(tm_plan_create(ctx.handle, st, len(steps), ctypes.byref(inp), ctypes.byref(sps),  # noqa: F821
                             ctypes.byref(fps), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None, timed=False):
        """Replays the plan's graph; with timed=True the graph that also records stage events."""
        fn = tm_plan_run_timed if timed else tm_plan_run  # noqa: F821
        check(fn(self.handle, _stream(stream)))

    def results(self, stream=None):
        r, bufs = _result_struct(self.caps[0], self.n_pairs, self.caps[1], self.n_steps, self.fwd_cap, self.tri)
        check(tm_plan_results(self.handle, ctypes.byref(r), _stream(stream)))  # noqa: F821
        return _collect(r, bufs)

    def info(self):
        a, b, c, d = (ctypes.c_int32() for _ in range(4))
        check(tm_plan_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),  # noqa: F821
                           ctypes.byref(d)))
        return dict(threads=a.value, lanes=b.value, ctas=c.value, kernels_per_run=d.value)

    def tuning(self):
        """The launch choices of the plan's fused form (tm_plan_get_tuning) as a dict."""
        t = L.tm_plan_tuning()
        check(tm_plan_get_tuning(self.handle, ctypes.byref(t)))  # noqa: F821
        return {f: getattr(t, f) for f, _ in t._fields_}

    def stage_times(self):
        """(search kernel, ingest, fusion, tail, dense blocks, prep) device milliseconds of the
        last run if it was timed (run(timed=True)); zeros otherwise.  The tail runs from the later
        of the search and fusion kernels' ends to the end of the run (each branch's offsets +
        copy of its own records, and the triangulation when on)."""
        ms = np.zeros(L.TM_PLAN_STAGES, np.float32)
        check(tm_plan_stage_times(self.handle, ms.ctypes.data))  # noqa: F821
        return tuple(float(x) for x in ms)

    def close(self):
        if self.handle:
            check(tm_plan_destroy(self.handle))  # noqa: F821
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching server (tm_server_*)."""

    def __init__(self, ctx, max_batch_requests=64, max_inflight_batches=3, queue_capacity=1 << 16,
                 evict_after=0, sp=None, fp=None, tri=None):
        self.ctx = ctx
        c = L.tm_server_config()
        tm_server_config_default(ctypes.byref(c))  # noqa: F821
        c.max_batch_requests, c.max_inflight_batches = max_batch_requests, max_inflight_batches
        c.queue_capacity, c.evict_after = queue_capacity, evict_after
        if sp is not None:
            c.search = sp.struct()
        if fp is not None:
            c.fuse = fp.struct()
        if tri is not None:  # triangulate every match (TriParams)
            c.triangulate, c.tri = 1, tri.struct()
        self.triangulate = tri is not None
        h = ctypes.c_void_p()
        check(tm_server_start(ctx.handle, ctypes.byref(c), ctypes.byref(h)))  # noqa: F821
        self.handle = h
        self.meta = {}

    def submit(self, kf_id, kf, nbrs, q_free=None, nbr_free=None, mps=None, fwd_mps=None, fwd_skip=None):
        """fwd_mps: the new keyframe's own map points, fused into every neighbour; fwd_skip: per
        neighbour a byte per forward map point (1 = that neighbour already observes it)."""
        keep = []
        r = L.tm_request()
        r.kf_id = int(kf_id)
        r.kf = keyframe_view(kf, keep)
        nb = np.ascontiguousarray(nbrs, np.uint64)
        r.nbr_ids, r.n_nbrs = (nb.ctypes.data if len(nb) else None), len(nb)
        qf = _host(q_free, np.uint8)
        if nbr_free is not None and isinstance(nbr_free, (list, tuple)):
            nbr_free = np.concatenate([np.asarray(m, np.uint8) for m in nbr_free]) if len(nbr_free) else None
        nf = _host(nbr_free, np.uint8)
        r.q_free, r.nbr_free = _ptr(qf), _ptr(nf)
        if nf is not None:
            r.nbr_free_bytes = int(nf.numel()) if hasattr(nf, "numel") else int(nf.size)
        r.mps = mappoint_view(mps if mps is not None and mps["n"] else None, keep)
        r.fwd_mps = mappoint_view(fwd_mps if fwd_mps is not None and fwd_mps["n"] else None, keep)
        if fwd_skip is not None and r.fwd_mps.n:
            fs = np.ascontiguousarray(np.concatenate([np.asarray(x, np.uint8).reshape(-1) for x in fwd_skip])
                                      if isinstance(fwd_skip, (list, tuple)) else np.asarray(fwd_skip, np.uint8))
            assert fs.size == len(nb) * r.fwd_mps.n
            keep.append(fs)
            r.fwd_skip = fs.ctypes.data
        t = ctypes.c_uint64()
        check(tm_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))  # noqa: F821
        self.meta[t.value] = (len(nb),)
        self.ctx.sizes[int(kf_id)] = r.kf.n
        return t.value

    def poll(self, ticket, timeout=0.0):
        info = L.tm_request_info()
        st = tm_server_poll(self.handle, ticket, float(timeout), ctypes.byref(info))  # noqa: F821
        if st not in (TM_OK, TM_ERR_TIMEOUT):
            check(st)
        return {f: getattr(info, f) for f, _ in info._fields_}

    def stats(self):
        """The server's counters since its start (tm_server_get_stats) as a dict: requests
        submitted / admitted / completed / failed, batches, admission rounds that waited for
        store memory (deferrals), keyframes evicted, and the peaks of the queue, of the batches
        in flight and of the store's occupied slots, beside the budget's slot limit."""
        st = L.tm_server_stats()
        check(tm_server_get_stats(self.handle, ctypes.byref(st)))  # noqa: F821
        return {f: getattr(st, f) for f, _ in st._fields_}

    def take(self, ticket):
        """Waits for the request and returns (per-pair match arrays, fusion array, info)."""
        info = self.poll(ticket, timeout=600.0)
        if not info["done"]:
            raise TMError(TM_ERR_TIMEOUT, "request %d not done" % ticket)
        n_nbrs = self.meta.pop(ticket)[0]
        m = np.zeros((max(1, info["n_matches"]), 3), np.int32)
        po = np.zeros(n_nbrs + 1, np.int32)
        f = np.zeros((max(1, info["n_fuse"]), 3), np.int32)
        check(tm_server_take(self.handle, ticket, m.ctypes.data, po.ctypes.data, f.ctypes.data))  # noqa: F821
        return _split(m[:info["n_matches"]], po), f[:info["n_fuse"]], info

    def take_ex(self, ticket):
        """Waits for the request; returns a dict: pairs (per neighbour), fuse, fwds (per
        neighbour), points and point_ok (None unless the server triangulates), info."""
        info = self.poll(ticket, timeout=600.0)
        if not info["done"]:
            raise TMError(TM_ERR_TIMEOUT, "request %d not done" % ticket)
        n_nbrs = self.meta.pop(ticket)[0]
        nm = info["n_matches"]
        m = np.zeros((max(1, nm), 3), np.int32)
        po = np.zeros(n_nbrs + 1, np.int32)
        f = np.zeros((max(1, info["n_fuse"]), 3), np.int32)
        fw = np.zeros((max(1, info["n_fwd"]), 3), np.int32)
        fo = np.zeros(n_nbrs + 1, np.int32)
        pts = np.zeros((max(1, nm), 3), np.float32) if self.triangulate else None
        ok = np.zeros(max(1, nm), np.uint8) if self.triangulate else None
        check(tm_server_take_ex(self.handle, ticket, m.ctypes.data, po.ctypes.data, f.ctypes.data,  # noqa: F821
                                fw.ctypes.data, fo.ctypes.data, _ptr(pts), _ptr(ok)))
        return dict(pairs=_split(m[:nm], po), fuse=f[:info["n_fuse"]], fwds=_split(fw[:info["n_fwd"]], fo),
                    points=None if pts is None else pts[:nm], point_ok=None if ok is None else ok[:nm], info=info)

    def close(self):
        if self.handle:
            check(tm_server_stop(self.handle))  # noqa: F821
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
