"""Host-side logic that needs no GPU: the random-search draws and the
synthetic anchor generator's structure."""
import numpy as np

from paper_1512_01641_gb300 import synth, tune


def test_random_draws_are_seeded_and_inside_their_ranges():
    a = tune.random_draws(50, seed=4)
    b = tune.random_draws(50, seed=4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(np.array(a), np.array(tune.random_draws(50, seed=5)))
    for th in a:
        assert np.array_equal(th[:4], tune.THETA0[:4])
        for k, (lo, hi) in tune.RANDOM_RANGES.items():
            assert lo <= th[tune._THETA_INDEX[k]] <= hi


def test_random_draws_of_a_subset_keep_the_other_parameters():
    for th in tune.random_draws(20, seed=1, ranges={"thr": (0.3, 0.4)}):
        assert th[4] == tune.THETA0[4] and th[5] == tune.THETA0[5]
        assert 0.3 <= th[6] <= 0.4


def test_anchor_lists_are_sorted_distinct_and_in_range():
    b = synth.make_batch(90, 12, planted_frac=0.5, size_median=20, size_hi=50)
    for a, n in zip(synth.make_anchors(b, 91, v_anchor=300, p_anchor=0.8, max_per=3),
                    (len(b.src.sent_tok_off) - 1, len(b.tgt.sent_tok_off) - 1)):
        assert len(a.sent_off) == n + 1 and a.sent_off[0] == 0 and a.sent_off[-1] == len(a.ids)
        assert np.all(np.diff(a.sent_off) >= 0) and np.all(np.diff(a.sent_off) <= 3)
        assert a.ids.min() >= 0 and a.ids.max() < 300
        for s in range(n):
            x = a.ids[a.sent_off[s]:a.sent_off[s + 1]]
            assert np.all(np.diff(x) > 0)
