"""The oracle's pins must catch plausible mistakes: each mutation below plants one bug in a
copy of the oracle's C source (on the CPU), or in its fuse-apply map, and at least one pin
must then fail."""

import os
import shutil

import pytest

import oracle as O
from tests import test_fuse_apply as FA
from tests import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "tm_oracle.c")

# (name, text in tm_oracle.c, replacement)
MUTATIONS = [
    ("hamming drops a bit", "bit < 8; ++bit", "bit < 7; ++bit"),
    ("epipolar sigma from query level", "thr[T->level[j]]", "thr[Q->level[i]]"),
    ("epipolar line from F, not F^T", "float a = (xq * F[0] + yq * F[3]) + F[6];",
     "float a = (xq * F[0] + yq * F[1]) + F[2];"),
    ("relative translation sign", "t[r] = tq[r] - s;", "t[r] = tq[r] + s;"),
    ("K^-1 uses cy for x", "-cam->cx / cam->fx", "-cam->cy / cam->fx"),
    ("R = R_T R_Q^T", "orc_mat3_mul(Rq, RtT, R);", "orc_mat3_mul(RtT, Rq, R);"),
    ("no second-best update on ties", "} else if (d < second) {", "} else if (d < second && d != best) {"),
    ("ratio test non-strict", "!((int64_t)p->ratio_den * best < (int64_t)p->ratio_num * second)",
     "!((int64_t)p->ratio_den * best <= (int64_t)p->ratio_num * second)"),
    ("Hamming threshold strict", "if (best > p->hamming_max) continue;", "if (best >= p->hamming_max) continue;"),
    ("resolve ties to the higher query", "if (win < 0 || acc_d[i] < acc_d[win]) win = i;",
     "if (win < 0 || acc_d[i] <= acc_d[win]) win = i;"),
    ("rotation bin 30 not folded", "if (bin >= ORC_BINS) bin = 0;", "if (bin >= ORC_BINS) bin = ORC_BINS - 1;"),
    ("rotation difference reversed", "float rot = angle_q - angle_t;", "float rot = angle_t - angle_q;"),
    ("top-3 ties to the higher bin", "if (bestb < 0 || hist[b] > hist[bestb]) bestb = b;",
     "if (bestb < 0 || hist[b] >= hist[bestb]) bestb = b;"),
    ("tenth rule non-strict", "10 * hist[top[r]] < mx", "10 * hist[top[r]] <= mx"),
    ("only the top-2 bins", "for (int r = 0; r < 3; ++r) {\n            int bestb", "for (int r = 0; r < 2; ++r) {\n            int bestb"),
    ("comparisons counted after the gate", "comparisons++;\n            int d = orc_hamming(Q->desc",
     "int d = orc_hamming(Q->desc"),
    ("fuse camera centre sign", "O[c] = (float)(-s);", "O[c] = (float)(s);"),
    ("fuse predicted level strict", "if (dist * scale[l] >= max_dist[m]) {", "if (dist * scale[l] > max_dist[m]) {"),
    ("fuse level window pl+1", "if (lv != pl && lv != pl - 1) continue;", "if (lv != pl && lv != pl + 1) continue;"),
    ("fuse radius from scale^2", "float r = p->radius_scale * scale[pl];", "float r = p->radius_scale * sigma2[pl];"),
    ("fuse viewing angle dropped", "if (cosv < 0.5f * dist) continue;", ""),
    ("fuse chi2 uses predicted level", "<= thr[lv])) continue;", "<= thr[pl])) continue;"),
    ("fuse ignores skip", "if (skip && skip[m]) continue;", ""),
    ("fuse u uses fy", "float u = fx * x + cx, v = fy * y + cy;", "float u = fy * x + cy, v = fy * y + cy;"),
    ("search ignores target mask", "if (free_t && !free_t[j]) continue;", ""),
    ("ORB bins floored", "(int)roundf(rot * (1.0f / 30.0f))", "(int)floorf(rot * (1.0f / 30.0f))"),
    ("epipole from the centre's mirror", "        cq[k] = -s;", "        cq[k] = s;"),
    ("epipole x uses cy", "e[0] = (float)(cam->fx * (c[0] / c[2]) + cam->cx);",
     "e[0] = (float)(cam->fx * (c[0] / c[2]) + cam->cy);"),
    ("baseline skip inverted", "if (base / (double)p->t_median_depth < (double)p->baseline_min_ratio) {",
     "if (base / (double)p->t_median_depth > (double)p->baseline_min_ratio) {"),
    ("midpoint parameter sign", "const float s1 = (b * e - c2 * d) / den", "const float s1 = (c2 * d - b * e) / den"),
    ("parallax bound dropped", "if (!(cosp > 0.0f && cosp < cos_max)) continue;", "if (!(cosp > 0.0f)) continue;"),
    ("reprojection in one view only",
     "        if (!orc_view_ok(cam, &V[1], X, u[1], vv[1], chi2 * sigma2[lev[1]])) continue;\n", ""),
    ("scale consistency dropped",
     "if (ratio_dist * f < ratio_octave || ratio_dist > ratio_octave * f) continue;", ""),
]

PINS = [
    P.test_ratio_golden, P.test_resolve_golden, P.test_rotation_golden, P.test_fuse_golden,
    lambda: P.test_hamming_argmin_brute_force(0), lambda: P.test_node_buckets_brute_force(1),
    lambda: P.test_fundamental_epipolar_constraint(0), lambda: P.test_epipolar_gate_geometric(0),
    lambda: P.test_planted_recovery(0), P.test_step_invariants,
    lambda: P.test_fuse_gates_geometric(0), P.test_fuse_planted, P.test_forward_fusion_skip_and_independence,
    P.test_orb_rotation_bins_golden, lambda: P.test_epipole_on_every_epipolar_line(0),
    P.test_epipole_rejection_invariants, P.test_triangulation_recovers_exact_points,
    P.test_triangulation_rejects_pure_rotation_and_scale_jumps, P.test_pair_baseline_skip,
    P.test_triangulation_parallax_bound_alone, P.test_triangulation_point_behind_second_view,
]


@pytest.fixture(scope="module")
def workdir():
    # the mutated copies are built beside the oracle, in its (git-ignored) build folder
    d = os.path.join(os.path.dirname(O.__file__), "_build", "mutations_%d" % os.getpid())
    os.makedirs(d, exist_ok=True)
    yield d
    O.use_library(None)
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(workdir, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(workdir, "mut_%d.c" % MUTATIONS.index((name, old, new)))
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = O.build(force=True, src=path, out=path[:-2] + ".so")
    O.use_library(lib)
    failed = []
    try:
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                failed.append(getattr(pin, "__name__", "pin"))
                break
    finally:
        O.use_library(None)
    assert failed, "no pin caught: " + name


# Mistakes planted in the fuse-apply map (plain Python), each a subclass overriding one step.
class _TieToExisting(O.FuseMap):
    def fuse(self, k, cands):  # a tie keeps the point already at the keypoint
        st = dict(added=0, merged_into_existing=0, replaced_existing=0, skipped_dead=0, skipped_observed=0)
        for m, j in cands:
            if m in self.replaced:
                st["skipped_dead"] += 1
            elif k in self.obs[m]:
                st["skipped_observed"] += 1
            elif self.kp[k][j] is None:
                self.observe(k, j, m)
                st["added"] += 1
            elif len(self.obs[self.kp[k][j]]) >= len(self.obs[m]):
                self._replace(m, self.kp[k][j])
                st["merged_into_existing"] += 1
            else:
                self._replace(self.kp[k][j], m)
                st["replaced_existing"] += 1
        return st


class _NoErase(O.FuseMap):
    def _replace(self, a, b):  # a keyframe that already sees b keeps its link to a
        for k, j in self.obs.pop(a).items():
            if k not in self.obs[b]:
                self.obs[b][k] = j
                self.kp[k][j] = b
        self.replaced[a] = b


class _NoDeadSkip(O.FuseMap):
    def fuse(self, k, cands):  # a replaced point stands for its survivor instead of being skipped
        st = dict(added=0, merged_into_existing=0, replaced_existing=0, skipped_dead=0, skipped_observed=0)
        for m, j in cands:
            m = self.current(m)
            if k in self.obs[m]:
                st["skipped_observed"] += 1
            elif self.kp[k][j] is None:
                self.observe(k, j, m)
                st["added"] += 1
            elif len(self.obs[self.kp[k][j]]) > len(self.obs[m]):
                self._replace(m, self.kp[k][j])
                st["merged_into_existing"] += 1
            else:
                self._replace(self.kp[k][j], m)
                st["replaced_existing"] += 1
        return st


@pytest.mark.parametrize("cls", [_TieToExisting, _NoErase, _NoDeadSkip], ids=lambda c: c.__name__)
def test_fuse_apply_mutation_is_caught(monkeypatch, cls):
    monkeypatch.setattr(O, "FuseMap", cls)
    with pytest.raises(AssertionError):
        FA.test_oracle_worked_case()
