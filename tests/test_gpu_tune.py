"""Tuning drivers (grid search and Adam on the soft alignment) on the GPU."""
import numpy as np
import pytest

from paper_1512_01641_gb300 import synth

pytestmark = pytest.mark.gpu


def _batches(n_train=300, n_eval=150):
    rng = np.random.Generator(np.random.PCG64(5))
    dic = synth.make_dictionary(rng, 5000, 5000)
    tr = synth.make_batch(501, n_train, dic=dic, planted_frac=1.0, p_ins=0.3, p_wdrop=0.25, size_median=30,
                          size_hi=120)
    ev = synth.make_batch(502, n_eval, dic=dic, planted_frac=1.0, p_ins=0.3, p_wdrop=0.25, size_median=30,
                          size_hi=120)
    return tr, ev


def test_link_gold_counts_match_host_count():
    from paper_1512_01641_gb300 import miner, tune
    tr, _ = _batches(80, 10)
    d = tune.TuneData(tr)
    params = miner.MineParams()
    res = d.f1(params)
    links = miner.links_per_pair(d.out, tr.n_pairs)
    tp = sum(len({(i, j) for i, j, _ in links[k]} & {tuple(x) for x in tr.gold[k].tolist()}) for k in range(tr.n_pairs))
    assert res["correct"] == tp
    assert res["links"] == sum(len(l) for l in links)
    assert res["gold"] == sum(len(g) for g in tr.gold)


def test_grid_search_picks_best_training_setting():
    from paper_1512_01641_gb300 import miner, tune
    tr, ev = _batches(120, 40)
    train, held = tune.TuneData(tr), tune.TuneData(ev)
    grid = {"gap": [0.1, 0.4], "thr": [0.3, 0.6], "b": [-4.0, -2.0]}
    r = tune.grid_search(train, held, grid=grid)
    best = -1
    for gap in grid["gap"]:
        for thr in grid["thr"]:
            for b in grid["b"]:
                th = tune.THETA0.copy()
                th[4], th[5], th[6] = b, gap, thr
                best = max(best, train.f1(miner.params_from_theta(th))["f1"])
    assert r.train_f1 == pytest.approx(best)


def test_adam_lowers_soft_loss():
    from paper_1512_01641_gb300 import tune
    tr, ev = _batches()
    train, held = tune.TuneData(tr), tune.TuneData(ev)
    r = tune.adam_tune(train, held, steps=30)
    assert r.extra["loss_last"] < r.extra["loss_first"]
    assert 0.0 < r.eval["f1"] <= 1.0


def test_random_search_keeps_the_best_draw_and_is_seeded():
    from paper_1512_01641_gb300 import miner, tune
    tr, ev = _batches(120, 40)
    train, held = tune.TuneData(tr), tune.TuneData(ev)
    r = tune.random_search(train, held, trials=12, seed=3)
    f1s = [train.f1(miner.params_from_theta(th))["f1"] for th in tune.random_draws(12, seed=3)]
    assert r.train_f1 == pytest.approx(max(f1s))
    assert r.theta == pytest.approx(tune.random_draws(12, seed=3)[int(np.argmax(f1s))].tolist())
    lo, hi = tune.RANDOM_RANGES["gap"]
    assert lo <= r.theta[5] <= hi
    # the paper's two-parameter form leaves b at its starting value
    r2 = tune.random_search(train, held, trials=4, seed=1, ranges={"gap": (0.1, 0.5), "thr": (0.3, 0.7)})
    assert r2.theta[4] == tune.THETA0[4]


def test_gpu_link_matches_equal_nw_similarity_of_link_lists():
    # the GPU's correct-link count is the oracle's Needleman-Wunsch alignment
    # of each pair's automatic and gold link lists (Section 5.2 reading)
    import oracle.evaluate as ev
    from paper_1512_01641_gb300 import miner, tune
    tr, _ = _batches(60, 10)
    d = tune.TuneData(tr)
    params = miner.MineParams(gap=0.2, thr=0.4)
    res = d.f1(params)
    links = miner.links_per_pair(d.out, tr.n_pairs)
    sim = ev.similarity([[(i, j) for i, j, _ in l] for l in links], [[tuple(x) for x in g.tolist()] for g in tr.gold])
    assert (res["correct"], res["links"], res["gold"]) == (sim["matched"], sim["auto"], sim["human"])
    assert res["f1"] == pytest.approx(sim["similarity"])
