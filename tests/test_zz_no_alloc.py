"""tm_search_pair_noalloc is the correspondence search for callers that cannot allocate device
memory (under a fixed memory budget, in a real-time loop that forbids allocation after
start-up, or without a context and its store): it keeps its scratch in one fixed array inside
the library.  Called twice in a row through the C ABI -- a 1200-keypoint pair with masks,
then a smaller 500-keypoint pair without, so that leftovers of the first call in the shared
array would show -- it must give exactly the matches and comparison count of
tm_search_triangulation and of the oracle.  Oversized keyframes, host memory and misaligned
arrays are refused before any work.

This file is collected last on purpose."""

import ctypes

import numpy as np
import pytest

from gen import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_equals_search_triangulation():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import oracle as O
    import paper_2511_02036_gb300 as tm
    from paper_2511_02036_gb300 import _lib as L

    w = W.make_cfg1(seed=1003)
    st = w["steps"][0]
    p = W.make_pair_cfg0(5)
    cases = [(w["cam"], w["frames"][st["q"]], w["frames"][st["nbrs"][0]], st["q_free"], st["nbr_free"][0]),
             (p["cam"], p["Q"], p["T"], None, None)]
    keep = []

    def dev(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        keep.append(t)
        return t

    def view(kf):
        v = L.tm_keyframe_view()
        v.n = int(kf["n"])
        v.desc, v.xy, v.angle, v.level, v.node = (
            dev(kf["desc"]).data_ptr(), dev(kf["xy"]).data_ptr(), dev(kf["angle"]).data_ptr(),
            dev(kf["level"]).data_ptr(), dev(kf["node"].view(np.int32)).data_ptr())
        v.Tcw[:] = [float(x) for x in np.asarray(kf["Tcw"], np.float64).reshape(12)]
        return v

    for cam, Q, T, fq, ft in cases:  # two calls in a row
        with tm.Context(cam, max_kp=2048) as ctx:
            ctx.add_keyframes([1, 2], [Q, T])
            exp, ecmp = ctx.search(1, [2], fq, None if ft is None else [ft])
        out = torch.full((Q["n"], 3), -1, dtype=torch.int32, device="cuda")
        n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
        ncmp = torch.zeros(1, dtype=torch.int64, device="cuda")
        c = tm.camera_struct(cam)
        qv, tv = view(Q), view(T)
        sp = tm.SearchParams().struct()
        st_ = tm.tm_search_pair_noalloc(ctypes.byref(c), ctypes.byref(qv), ctypes.byref(tv),
                                        ctypes.byref(sp),
                                        None if fq is None else dev(fq).data_ptr(),
                                        None if ft is None else dev(ft).data_ptr(),
                                        out.data_ptr(), n_out.data_ptr(), ncmp.data_ptr(), None)
        assert st_ == tm.TM_OK, tm._clib.tm_last_error()
        torch.cuda.synchronize()
        n = int(n_out.item())
        np.testing.assert_array_equal(out[:n].cpu().numpy(), exp[0])
        assert int(ncmp.item()) == ecmp
        assert n == len(exp[0]) and n > 50
        # and the oracle's, directly
        om, ocmp = O.search_pair(cam, Q, T, fq, ft)
        np.testing.assert_array_equal(out[:n].cpu().numpy(), om)
        assert int(ncmp.item()) == ocmp

    # arguments the kernels could not read safely are refused before any work: a descriptor
    # array 8 bytes off its 16-byte alignment, keyframe arrays in host memory
    cam, Q, T = cases[1][0], cases[1][1], cases[1][2]
    c = tm.camera_struct(cam)
    out = torch.zeros((Q["n"], 3), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    qv, tv = view(Q), view(T)
    bad = L.tm_keyframe_view.from_buffer_copy(qv)
    padded_desc = dev(np.zeros((Q["n"] + 1) * 32, np.uint8))
    bad.desc = padded_desc.data_ptr() + 8
    st_ = tm.tm_search_pair_noalloc(ctypes.byref(c), ctypes.byref(bad), ctypes.byref(tv), None, None, None,
                                    out.data_ptr(), n_out.data_ptr(), None, None)
    assert st_ == tm.TM_ERR_INVALID_ARG
    assert b"aligned" in tm._clib.tm_last_error()
    host_desc = np.ascontiguousarray(Q["desc"])
    bad.desc = host_desc.ctypes.data
    st_ = tm.tm_search_pair_noalloc(ctypes.byref(c), ctypes.byref(bad), ctypes.byref(tv), None, None, None,
                                    out.data_ptr(), n_out.data_ptr(), None, None)
    assert st_ == tm.TM_ERR_INVALID_ARG

    # beyond the fixed scratch size: refused before any work
    big = W.random_keyframe(np.random.default_rng(0), L.TM_MAX_KP_LIMIT, W.CAM_CFG0)
    big["n"] = 2049
    c = tm.camera_struct(W.CAM_CFG0)
    v = view(dict(big, desc=big["desc"][:2049], xy=big["xy"][:2049], angle=big["angle"][:2049],
                  level=big["level"][:2049], node=big["node"][:2049]))
    out = torch.zeros((2049, 3), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st_ = tm.tm_search_pair_noalloc(ctypes.byref(c), ctypes.byref(v), ctypes.byref(v), None, None, None,
                                    out.data_ptr(), n_out.data_ptr(), None, None)
    assert st_ == tm.TM_ERR_INVALID_ARG
    assert b"2048" in tm._clib.tm_last_error()
