"""Wave planner of the sweep split along the channel (host logic, no GPU): consecutive split
items share a wave while their staging fits the cap, and the record buffer is sized by the
most records any wave of the partition in use holds.  That figure is not monotonic in the
cap, so a partition re-made under an HBM budget must be sized on its own."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def negf():
    from paper_2407_14633_gb300 import build
    build.build()
    from paper_2407_14633_gb300 import negf as m
    m.load()
    return m


def brute_force(stage, n_seg, cap):
    """The same greedy rule written out: a new wave starts when the next item would push the
    current wave's staging over the cap (a wave always takes at least one item)."""
    waves, cur, st = [], [], 0
    for i, b in enumerate(stage):
        if cur and st + b > cap:
            waves.append(cur)
            cur, st = [], 0
        cur.append(i)
        st += b
    if cur:
        waves.append(cur)
    wave_of = np.zeros(len(stage), dtype=np.int32)
    for w, items in enumerate(waves):
        wave_of[items] = w
    max_stage = max((sum(stage[i] for i in w) for w in waves), default=0)
    max_rec = max((sum(n_seg[i] for i in w) for w in waves), default=0)
    return wave_of, max_stage, max_rec


def test_records_of_the_largest_wave_grow_when_the_cap_shrinks(negf):
    # (staging, records): a long real-axis item, two contour items, a short real-axis item
    stage, n_seg = [45, 40, 40, 6], [15, 20, 20, 2]
    w90, s90, r90 = negf.plan_seg_waves(stage, n_seg, 90)
    w80, s80, r80 = negf.plan_seg_waves(stage, n_seg, 80)
    assert list(w90) == [0, 0, 1, 1] and (s90, r90) == (85, 35)
    assert list(w80) == [0, 1, 1, 2] and (s80, r80) == (80, 40)
    assert r80 > r90   # sizing by the larger cap's partition would be too small


def test_partition_matches_the_greedy_rule(negf):
    rng = np.random.default_rng(11)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        L = rng.integers(16384, 200000, n)
        kind = rng.integers(0, 2, n)                       # 0 real axis (3 fields), 1 contour (2)
        stage = (L * np.where(kind == 0, 3, 2) * 32 * 8).astype(np.int64)
        n_seg = ((L + 511) // 512).astype(np.int32)
        cap = int(rng.integers(stage.min() // 2, stage.sum() + 2))
        got = negf.plan_seg_waves(stage, n_seg, cap)
        want = brute_force(list(stage), list(n_seg), cap)
        assert np.array_equal(got[0], want[0]) and got[1:] == want[1:], trial
        # every wave of more than one item fits the cap; waves are consecutive
        assert np.all(np.diff(got[0]) >= 0) and np.all(np.diff(got[0]) <= 1)
        for w in np.unique(got[0]):
            sel = got[0] == w
            assert sel.sum() == 1 or stage[sel].sum() <= cap


def test_oversize_item_forms_its_own_wave(negf):
    wave, st, rec = negf.plan_seg_waves([10, 500, 10], [1, 7, 1], 100)
    assert list(wave) == [0, 1, 2] and st == 500 and rec == 7


def test_invalid_arguments(negf):
    with pytest.raises(negf.NegfError):
        negf.plan_seg_waves([10], [0], 100)
    with pytest.raises(negf.NegfError):
        negf.plan_seg_waves([-1], [1], 100)
    assert negf.plan_seg_waves([], [], 100)[1:] == (0, 0)
