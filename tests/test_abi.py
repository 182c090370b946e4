"""The C-ABI library loads and exports every function include/*.h declares, and the Python
binding's structs have the C layout (no GPU needed: no compute call is made)."""

import ctypes
import glob
import os
import re
import shutil
import subprocess

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tm_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2511_02036_gb300 import _lib
    return _lib.load()


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only",
                          os.path.join(ROOT, "paper_2511_02036_gb300", "libtm.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None
    from paper_2511_02036_gb300 import _lib as L
    assert set(L.SIGNATURES) == set(names)


def test_struct_layout_matches_c(lib):
    from paper_2511_02036_gb300 import _lib as L
    structs = ["tm_camera", "tm_keyframe_view", "tm_mappoint_view", "tm_search_params",
               "tm_fuse_params", "tm_match", "tm_store_stats", "tm_step", "tm_batch_inputs",
               "tm_batch_result", "tm_server_config", "tm_request", "tm_request_info", "tm_fuse_apply_stats",
               "tm_plan_tuning", "tm_server_stats", "tm_keyframes_packed"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tm.h"', "int main(void){"]
    for s in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in getattr(L, s)._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0;}")
    # the probe program is built in the tests' own (git-ignored) build folder
    d = os.path.join(ROOT, "tests", "_build", "abi_%d" % os.getpid())
    os.makedirs(d, exist_ok=True)
    try:
        c = os.path.join(d, "abi.c")
        open(c, "w").write("\n".join(lines))
        exe = os.path.join(d, "abi")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    finally:
        shutil.rmtree(d, ignore_errors=True)
    got = dict(ln.split() for ln in out.splitlines())
    for s in structs:
        T = getattr(L, s)
        assert int(got[s]) == ctypes.sizeof(T), s
        for f, _ in T._fields_:
            assert int(got["%s.%s" % (s, f)]) == getattr(T, f).offset, (s, f)


def test_parameter_defaults(lib):
    from paper_2511_02036_gb300 import _lib as L
    import paper_2511_02036_gb300 as tm
    p = L.tm_search_params()
    lib.tm_search_params_default(ctypes.byref(p))
    assert (p.hamming_max, p.ratio_num, p.ratio_den, p.epipolar, p.resolve, p.rot_filter) == (50, 3, 5, 1, 1, 1)
    assert abs(p.epi_chi2 - 3.84) < 1e-6 and p.mode == tm.TM_MODE_FUSED and p.lanes_per_query == 0
    f = L.tm_fuse_params()
    lib.tm_fuse_params_default(ctypes.byref(f))
    assert abs(f.chi2 - 5.99) < 1e-6 and f.hamming_max == 50 and f.radius_scale == 3.0
    # the Python defaults mirror the C defaults
    s = tm.SearchParams().struct()
    for k, _ in L.tm_search_params._fields_:
        if k != "epi_chi2":
            assert getattr(s, k) == getattr(p, k), k
    # the ORB-family preset and its coarse mode differ from the defaults only where stated
    o, oc = tm.SearchParams.orb_family().struct(), tm.SearchParams.orb_family(coarse=True, mode=1).struct()
    assert (o.epipole_px, o.rot_mode, o.epipolar) == (10.0, 1, 1) and abs(o.baseline_min_ratio - 0.01) < 1e-9
    assert (oc.epipolar, oc.epipole_px, oc.rot_mode, oc.mode) == (0, 10.0, 1, 1)
    for k, _ in L.tm_search_params._fields_:
        if k not in ("epi_chi2", "epipole_px", "rot_mode", "baseline_min_ratio"):
            assert getattr(o, k) == getattr(p, k), k


def test_null_arguments_rejected(lib):
    from paper_2511_02036_gb300 import _lib as L
    # argument checks happen before any CUDA call
    assert lib.tm_ctx_create(0, None, 100, 0, None) == L.TM_ERR_INVALID_ARG
    assert lib.tm_ctx_destroy(None) == L.TM_ERR_INVALID_ARG
    assert lib.tm_plan_run(None, None) == L.TM_ERR_INVALID_ARG
    assert b"null" in lib.tm_last_error()
    cam = L.tm_camera(640, 480, 450.0, 450.0, 320.0, 240.0)
    h = ctypes.c_void_p()
    assert lib.tm_ctx_create(0, ctypes.byref(cam), 0, 0, ctypes.byref(h)) == L.TM_ERR_INVALID_ARG
    assert lib.tm_ctx_create(0, ctypes.byref(cam), L.TM_MAX_KP_LIMIT + 1, 0, ctypes.byref(h)) == L.TM_ERR_INVALID_ARG
    wide = L.tm_camera(L.TM_MAX_IMAGE_SIZE + 1, 480, 450.0, 450.0, 320.0, 240.0)
    assert lib.tm_ctx_create(0, ctypes.byref(wide), 100, 0, ctypes.byref(h)) == L.TM_ERR_INVALID_ARG


def test_struct_arrays_match_ctypes_layout():
    """The binding fills arrays of C records through numpy structured views; each field must
    land where the ctypes (and C) layout puts it."""
    import paper_2511_02036_gb300 as tm
    from paper_2511_02036_gb300 import _lib as L
    keep = []
    kfs = [dict(desc=np.zeros((3, 32), np.uint8), xy=np.zeros((3, 2), np.float32),
                angle=np.zeros(3, np.float32), level=np.zeros(3, np.uint8),
                node=np.arange(3, dtype=np.uint32), Tcw=np.arange(12, dtype=np.float64) + 10 * k)
           for k in range(2)]
    v = tm.keyframe_views(kfs, keep)
    for k in range(2):
        c = L.tm_keyframe_view.from_address(v.ctypes.data + k * ctypes.sizeof(L.tm_keyframe_view))
        assert c.n == 3 and c.node == kfs[k]["node"].ctypes.data and c.desc == kfs[k]["desc"].ctypes.data
        assert list(c.Tcw) == list(kfs[k]["Tcw"])
    steps = [dict(kf_id=5, nbrs=[1, 2], q_free_off=7, nbr_free_off=9, mp_begin=3, mp_count=4),
             dict(kf_id=6, nbrs=[], mp_count=0)]
    ctx = tm.Context.__new__(tm.Context)
    ctx.sizes = {}
    st, inp, keep2 = ctx._inputs(steps, masks=np.zeros(16, np.uint8),
                                 mps=dict(n=0, pos=None, normal=None, desc=None, min_dist=None, max_dist=None))
    c0 = L.tm_step.from_address(st)
    c1 = L.tm_step.from_address(st + ctypes.sizeof(L.tm_step))
    assert (c0.kf_id, c0.n_nbrs, c0.q_free_off, c0.nbr_free_off, c0.mp_begin, c0.mp_count) == (5, 2, 7, 9, 3, 4)
    assert list((ctypes.c_uint64 * 2).from_address(c0.nbr_ids)) == [1, 2]
    assert (c1.kf_id, c1.n_nbrs, c1.q_free_off, c1.mp_count) == (6, 0, -1, 0)
    # result capacities: sum over pairs of min(n_Q, n_T)
    assert tm._result_caps([dict(kf_id=1, nbrs=[2, 3]), dict(kf_id=2, nbrs=[1])], {1: 10, 2: 4, 3: 20}) == (4 + 10 + 4, 0)


def test_packed_keyframe_views():
    """Keyframes packed one after another in one array per field give the same records as the
    per-keyframe form (pointers at each keyframe's first element)."""
    import paper_2511_02036_gb300 as tm
    from paper_2511_02036_gb300 import _lib as L
    rng = np.random.default_rng(0)
    ns = [3, 0, 5]
    N = sum(ns)
    packed = dict(n=ns, desc=rng.integers(0, 255, (N, 32), dtype=np.uint8), xy=rng.random((N, 2), np.float32),
                  angle=rng.random(N, np.float32), level=rng.integers(0, 8, N, dtype=np.uint8),
                  node=rng.integers(0, 99, N, dtype=np.uint32), Tcw=rng.random((3, 12)))
    keep = []
    v = tm.keyframe_views_packed(packed, keep)
    off = 0
    for k, n in enumerate(ns):
        c = L.tm_keyframe_view.from_address(v.ctypes.data + k * ctypes.sizeof(L.tm_keyframe_view))
        assert c.n == n and list(c.Tcw) == list(packed["Tcw"][k])
        if n:
            assert c.desc == packed["desc"].ctypes.data + 32 * off
            assert c.xy == packed["xy"].ctypes.data + 8 * off
            assert c.node == packed["node"].ctypes.data + 4 * off
            assert c.level == packed["level"].ctypes.data + off
        else:
            assert c.desc is None or c.desc == 0
        off += n


def test_packed_keyframes_record():
    """keyframes_packed: one tm_keyframes_packed record pointing at the packed arrays (counts
    and poses converted to int32 / float64), and batch inputs that carry it instead of views."""
    import paper_2511_02036_gb300 as tm
    from paper_2511_02036_gb300 import _lib as L
    rng = np.random.default_rng(1)
    ns = [4, 0, 2]
    N = sum(ns)
    packed = dict(n=ns, desc=rng.integers(0, 255, (N, 32), dtype=np.uint8), xy=rng.random((N, 2), np.float32),
                  angle=rng.random(N, np.float32), level=rng.integers(0, 8, N, dtype=np.uint8),
                  node=rng.integers(0, 99, N, dtype=np.uint32), Tcw=rng.random((3, 3, 4)))
    keep = []
    p, counts = tm.keyframes_packed(packed, keep)
    assert list(counts) == ns and counts.dtype == np.int32
    assert list((ctypes.c_int32 * 3).from_address(p.n)) == ns
    assert list((ctypes.c_double * 36).from_address(p.Tcw)) == list(packed["Tcw"].reshape(36))
    assert (p.desc, p.xy, p.angle, p.level, p.node) == tuple(packed[k].ctypes.data for k in
                                                             ("desc", "xy", "angle", "level", "node"))

    class FakeCtx(tm.Context):
        def __init__(self):
            self.sizes, self._res, self.max_kp = {}, None, 2048
    ctx = FakeCtx()
    st, inp, keep2 = ctx._inputs([dict(kf_id=1, nbrs=[])], masks=np.zeros(1, np.uint8),
                                 mps=dict(n=0), new=([10, 11, 12], packed))
    assert inp.n_new == 3 and not inp.new_kfs and inp.new_packed
    rec = L.tm_keyframes_packed.from_address(inp.new_packed)
    assert rec.desc == packed["desc"].ctypes.data and list((ctypes.c_int32 * 3).from_address(rec.n)) == ns
    assert ctx.sizes == {10: 4, 11: 0, 12: 2}


def test_step_table_records_match_step_dicts():
    """StepTable.records gives the same tm_step records as the dict path (pointers aside)."""
    import paper_2511_02036_gb300 as tm
    steps = [dict(kf_id=7, nbrs=[1, 2, 3], q_free_off=0, nbr_free_off=10, mp_begin=0, mp_count=5),
             dict(kf_id=8, nbrs=[], q_free_off=-1, nbr_free_off=-1, mp_begin=5, mp_count=0),
             dict(kf_id=9, nbrs=[4], mp_begin=5, mp_count=2)]
    keep = []
    t = tm.StepTable.from_steps(steps)
    rec = t.records(keep)
    assert len(t) == 3 and list(t.nbr_ids) == [1, 2, 3, 4]
    assert list(rec["kf_id"]) == [7, 8, 9] and list(rec["n_nbrs"]) == [3, 0, 1]
    assert list(rec["q_free_off"]) == [0, -1, -1] and list(rec["nbr_free_off"]) == [10, -1, -1]
    assert list(rec["mp_begin"]) == [0, 5, 5] and list(rec["mp_count"]) == [5, 0, 2]
    nb = keep[0]
    assert rec["nbr_ids"][0] == nb.ctypes.data and rec["nbr_ids"][1] == 0
    assert rec["nbr_ids"][2] == nb.ctypes.data + 8 * 3
    mc, fc = tm._result_caps(t, {7: 100, 8: 50, 9: 10})
    assert mc == 100 * 3 + 10 * 1 and fc == 7


def test_pack_batch_forward_fusion_ranges():
    """Forward map points follow the step's own map points in the batch arrays; their skip
    bytes follow the step's masks, neighbour-major."""
    import paper_2511_02036_gb300 as tm
    mp = lambda n, v: dict(n=n, pos=np.full((n, 3), v, np.float32), normal=np.zeros((n, 3), np.float32),  # noqa: E731
                           desc=np.zeros((n, 32), np.uint8), min_dist=np.zeros(n, np.float32),
                           max_dist=np.ones(n, np.float32), skip=np.zeros(n, np.uint8))
    steps = [dict(kf_id=1, nbrs=[2, 3], q_free=np.ones(4, np.uint8), nbr_free=[np.ones(5, np.uint8), np.ones(6, np.uint8)],
                  mps=mp(7, 1.0), fwd_mps=mp(3, 2.0), fwd_skip=[np.array([1, 0, 0], np.uint8), np.array([0, 0, 1], np.uint8)]),
             dict(kf_id=4, nbrs=[2], mps=mp(2, 3.0))]
    st, masks, mps, _keep = tm.pack_batch(steps, {1: 4, 2: 5, 3: 6, 4: 8})
    assert (st[0].mp_begin, st[0].mp_count, st[0].fwd_mp_begin, st[0].fwd_mp_count) == (0, 7, 7, 3)
    assert (st[1].mp_begin, st[1].mp_count, st[1].fwd_mp_count, st[1].fwd_skip_off) == (10, 2, 0, -1)
    assert st[0].q_free_off == 0 and st[0].nbr_free_off == 4 and st[0].fwd_skip_off == 15
    assert list(masks[15:21]) == [1, 0, 0, 0, 0, 1] and len(masks) == 21
    assert mps["n"] == 12 and mps["pos"][7, 0] == 2.0 and mps["pos"][10, 0] == 3.0
    assert tm._fwd_cap(steps) == 3 * 2


def test_normal_build_has_no_bounds_checks(lib):
    """tm_debug_bounds in the normal build: checks off, nothing recorded (no GPU call)."""
    site, en = ctypes.c_uint32(7), ctypes.c_int32(7)
    assert lib.tm_debug_bounds(1, ctypes.byref(site), ctypes.byref(en)) == 0
    assert (site.value, en.value) == (0, 0)
