"""How many epipolar-gate decisions lie near the threshold, and how many would change if the
gate were evaluated in float64 (an FP64 shadow of the float32 reading that both the oracle and
the GPU follow, bit for bit).  The gate (Sec. IV-C: a candidate must lie near the epipolar line
of its query) is taken in float32: line (a, b, c) = F^T x_Q, num = (a x_T + b y_T) + c,
pass iff num^2 < 3.84 sigma^2(level_T) (a^2 + b^2).  The shadow takes F, the line and the test
in float64.  Disagreements must be rare and lie close to the threshold (float32 rounding of F
and of the line, amplified by the cancellation in num, moves the decision value by a few
parts in 1e5 at most); the counts are printed (pytest -s)."""

import numpy as np
import pytest

import oracle as O
from gen import workloads as W


def f64_fundamental(cam, Tq, Tt):
    """F in float64 with x_Q^T F x_T = 0: K^-T [t]x R K^-1, R = R_Q R_T^T, t = t_Q - R t_T."""
    Tq = np.asarray(Tq, np.float64).reshape(3, 4)
    Tt = np.asarray(Tt, np.float64).reshape(3, 4)
    R = Tq[:, :3] @ Tt[:, :3].T
    t = Tq[:, 3] - R @ Tt[:, 3]
    tx = np.array([[0, -t[2], t[1]], [t[2], 0, -t[0]], [-t[1], t[0], 0]])
    K = np.array([[cam["fx"], 0, cam["cx"]], [0, cam["fy"], cam["cy"]], [0, 0, 1.0]])
    Ki = np.linalg.inv(K)
    return Ki.T @ tx @ R @ Ki


def thresholds32():
    s = [np.float32(1.0)]
    for _ in range(7):
        s.append(np.float32(s[-1] * np.float32(1.2)))
    return np.array([np.float32(3.84) * (x * x) for x in s], np.float32)


def candidates(Q, T):
    """Every same-node (query, target) pair: the comparisons the search makes, masks aside."""
    nq, nt = np.asarray(Q["node"]), np.asarray(T["node"])
    order = np.argsort(nt, kind="stable")
    lo = np.searchsorted(nt[order], nq, "left")
    hi = np.searchsorted(nt[order], nq, "right")
    qi = np.repeat(np.arange(len(nq)), hi - lo)
    tj = order[np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)])] if len(qi) else qi
    return qi, tj


def pairs_of(w, n_steps):
    for st in w["steps"][:n_steps]:
        for f in st["nbrs"]:
            yield w["frames"][st["q"]], w["frames"][f]


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg3"])
def test_gate_decisions_near_threshold(name):
    w = {"cfg1": W.make_cfg1, "cfg2": W.make_cfg2, "cfg3": W.make_cfg3}[name]()
    cam = w["cam"]
    thr32 = thresholds32()
    total = disagree = near5 = near4 = 0
    worst = 0.0
    for Q, T in pairs_of(w, 16):
        F32 = O.fundamental(cam, Q["Tcw"], T["Tcw"]).astype(np.float32)
        F64 = f64_fundamental(cam, Q["Tcw"], T["Tcw"])
        # the oracle's float32 F is the float64 F rounded (entrywise, within an ulp or two)
        np.testing.assert_allclose(F32, F64.astype(np.float32), rtol=3e-7, atol=0)
        qi, tj = candidates(Q, T)
        xq = np.asarray(Q["xy"], np.float32)[qi]
        xt = np.asarray(T["xy"], np.float32)[tj]
        lv = np.asarray(T["level"])[tj]
        # float32, in the reading's order, no contraction (numpy float32 ops round each step)
        a = (xq[:, 0] * F32[0, 0] + xq[:, 1] * F32[1, 0]) + F32[2, 0]
        b = (xq[:, 0] * F32[0, 1] + xq[:, 1] * F32[1, 1]) + F32[2, 1]
        c = (xq[:, 0] * F32[0, 2] + xq[:, 1] * F32[1, 2]) + F32[2, 2]
        num = (a * xt[:, 0] + b * xt[:, 1]) + c
        den = a * a + b * b
        d32 = (den > 0) & (num * num < thr32[lv] * den)
        # the float64 shadow
        x64, t64 = xq.astype(np.float64), xt.astype(np.float64)
        a6 = x64[:, 0] * F64[0, 0] + x64[:, 1] * F64[1, 0] + F64[2, 0]
        b6 = x64[:, 0] * F64[0, 1] + x64[:, 1] * F64[1, 1] + F64[2, 1]
        c6 = x64[:, 0] * F64[0, 2] + x64[:, 1] * F64[1, 2] + F64[2, 2]
        n6 = a6 * t64[:, 0] + b6 * t64[:, 1] + c6
        dn6 = a6 * a6 + b6 * b6
        th6 = 3.84 * 1.2 ** (2.0 * lv)
        d64 = n6 * n6 < th6 * dn6
        rel = np.abs(n6 * n6 / (th6 * dn6) - 1.0)
        total += len(qi)
        near5 += int((rel < 1e-5).sum())
        near4 += int((rel < 1e-4).sum())
        diff = d32 != d64
        disagree += int(diff.sum())
        if diff.any():
            worst = max(worst, float(rel[diff].max()))
    print("%s epipolar gate: %d decisions, %d within 1e-5 and %d within 1e-4 relative of the threshold, "
          "%d differ from the float64 shadow (largest relative margin of a difference %.2e)"
          % (name, total, near5, near4, disagree, worst))
    assert total > 5000
    assert disagree <= max(3, total // 10000)
    assert worst < 1e-4
    assert near4 < total // 1000
