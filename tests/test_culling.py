"""Keyframe-culling observation counters (host-side C in the library) against the list-walking
definition in the oracle, on random observation histories with insertions and removals."""

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def tm():
    import __graft_entry__ as g
    g.build()
    import paper_2511_02036_gb300 as tm
    return tm


@pytest.mark.parametrize("seed", range(4))
def test_counters_match_observation_lists(tm, seed):
    rng = np.random.default_rng(seed)
    n_mp, n_kf = 300, 40
    obs = {m: [] for m in range(n_mp)}           # map point -> [(keyframe, level)]
    with tm.ObsCounter(n_mp) as c:
        for kf in range(n_kf):
            mps = rng.choice(n_mp, size=int(rng.integers(20, 120)), replace=False)
            lv = rng.integers(0, 8, len(mps)).astype(np.uint8)
            for m, l in zip(mps, lv):
                obs[int(m)].append((kf, int(l)))
            c.add(mps, lv)
            if kf % 7 == 6:  # a keyframe culled: its observations removed
                gone = int(rng.integers(0, kf))
                ms = [m for m in range(n_mp) for (k, _) in obs[m] if k == gone]
                ls = [l for m in range(n_mp) for (k, l) in obs[m] if k == gone]
                c.remove(ms, ls)
                for m in ms:
                    obs[m] = [(k, l) for (k, l) in obs[m] if k != gone]
        for kf in range(n_kf):
            ms = [m for m in range(n_mp) for (k, _) in obs[m] if k == kf]
            ls = [l for m in range(n_mp) for (k, l) in obs[m] if k == kf]
            for th, ratio in ((3, 0.9), (1, 0.5), (5, 0.2)):
                got = c.redundant(ms, ls, th, ratio)
                assert got == O.culling_redundant(obs, kf, th, ratio), (kf, th, ratio)


def test_counter_errors(tm):
    with tm.ObsCounter(10) as c:
        c.add([1, 1, 2], [0, 0, 3])
        with pytest.raises(tm.TMError) as e:
            c.remove([1, 1, 1], [0, 0, 0])        # only two to remove: nothing removed
        assert e.value.status == tm.TM_ERR_NOT_FOUND
        # nothing was removed: map point 1 keeps both level-0 observations (one other besides
        # the keyframe's own), map point 2 has only the keyframe's own
        assert c.redundant([1], [0], th_obs=1) == (1, True)
        assert c.redundant([2], [3], th_obs=1) == (0, False)
        with pytest.raises(tm.TMError) as e:
            c.add([10], [0])
        assert e.value.status == tm.TM_ERR_INVALID_ARG
        with pytest.raises(tm.TMError):
            c.add([0], [8])
