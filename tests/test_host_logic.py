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


def test_noalloc_timeout_sentinel_is_reported():
    # the allocation-free entry point has no plan to record a device-side
    # timeout: it writes n_links = -1 and a NaN score, which the binding
    # turns into MINE_ETIMEOUT
    import math

    import pytest

    from paper_1512_01641_gb300 import miner
    assert miner.noalloc_result(3, 1.25) == (3, 1.25)
    assert miner.noalloc_result(0, -0.6) == (0, -0.6)
    with pytest.raises(miner.MinerError) as e:
        miner.noalloc_result(-1, math.nan)
    assert e.value.code == miner.MINE_ETIMEOUT
    with pytest.raises(miner.MinerError) as e:
        miner.noalloc_result(-2, 0.0)
    assert e.value.code == miner.MINE_EINVAL


def test_thin_dictionary_keeps_a_share_of_each_list():
    rng = np.random.Generator(np.random.PCG64(3))
    dic = synth.make_dictionary(rng, 3000, 3000)
    thin = synth.thin_dictionary(dic, 0.3, seed=4)
    assert thin.off[0] == 0 and thin.off[-1] == len(thin.tgt) and np.all(np.diff(thin.off) >= 0)
    kept = len(thin.tgt) / len(dic.tgt)
    assert 0.66 < kept < 0.74
    for v in rng.choice(3000, 50, replace=False):  # a subset of the original list, still sorted
        a, b = set(dic.translations(v).tolist()), thin.translations(v).tolist()
        assert set(b) <= a and b == sorted(b)
    assert np.array_equal(synth.thin_dictionary(dic, 0.3, seed=4).tgt, thin.tgt)
