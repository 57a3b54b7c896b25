"""GPU parity of the unconstrained (Yalign A*) aligner against the FP64
oracle (oracle/unconstrained.py), through the C ABI.

Tolerances: the pair score within 1e-5 * max(1, |A|); the matched cells
identical, except pairs whose GPU choice, re-scored in FP64 by the oracle's
cost model, lies within 1e-4 of the optimum (near ties, counted); links kept
at the threshold identical except cells within 1e-6 of it."""
import numpy as np
import pytest

import oracle
from oracle import unconstrained
from paper_1512_01641_gb300 import synth

from gpu_parity import H_REL, THR_BAND, TIE_TOL

pytestmark = pytest.mark.gpu


def _batch():
    # planted and unplanted pairs, sizes around the 32-column chunk edges,
    # single rows and columns
    ns = [1, 1, 5, 31, 33, 40, 12, 64, 3, 20]
    ms = [1, 9, 1, 33, 31, 45, 65, 30, 40, 20]
    dic = synth.make_dictionary(np.random.Generator(np.random.PCG64(700)), 800, 800)
    a = synth.make_batch(701, len(ns), dic=dic, planted_frac=0.0, src_sizes=ns, tgt_sizes=ms)
    b = synth.make_batch(702, 14, dic=dic, planted_frac=1.0, size_median=25, size_hi=60)
    return synth.concat_batches(a, b)


def _gpu(batch, params):
    import torch
    from paper_1512_01641_gb300 import miner
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    out = plan.align_unconstrained(params, counts)
    nw = plan.align(params, counts)
    torch.cuda.synchronize()
    return {"score": out["pair_score"].cpu().numpy()[:batch.n_pairs],
            "links": miner.links_per_pair(out, batch.n_pairs),
            "nw_score": nw["pair_score"].cpu().numpy()[:batch.n_pairs]}


def test_unconstrained_vs_oracle():
    from paper_1512_01641_gb300 import miner
    batch = _batch()
    p_all, p = miner.MineParams(thr=-1.0), miner.MineParams(thr=0.5)
    g_all, g = _gpu(batch, p_all), _gpu(batch, p)
    ref = oracle.mine(batch, p.w, p.b, p.gap, p.thr, want_sim=True)
    ties = 0
    for k in range(batch.n_pairs):
        s = ref["sim"][k]
        score, links = unconstrained.align(s, p.gap)
        for gg in (g_all, g):
            assert abs(gg["score"][k] - score) <= H_REL * max(1.0, abs(score)), (k, gg["score"][k], score)
        path = [(i, j) for i, j, _ in g_all["links"][k]]
        if path != links:  # several optimal choices: the GPU's must score within TIE_TOL of the optimum
            choice = [None] * s.shape[0]
            for i, j in path:
                choice[i] = j
            assert unconstrained.path_score(s, p.gap, choice) >= score - TIE_TOL, (k, path, links)
            ties += 1
        # at the threshold: the GPU path's cells with s >= thr, except inside the band
        kept = [(i, j) for i, j, _ in g["links"][k]]
        want = [(i, j) for i, j in path if s[i, j] >= p.thr]
        diff = set(kept) ^ set(want)
        assert all(abs(s[i, j] - p.thr) <= THR_BAND for i, j in diff), (k, sorted(diff))
        assert all(sv >= p.thr for _, _, sv in g["links"][k])
    assert ties <= max(2, batch.n_pairs // 6), ties
    # the move back only adds alignments: never worse than Needleman-Wunsch
    assert np.all(g["score"] >= g["nw_score"] - 1e-4 * np.maximum(1.0, np.abs(g["nw_score"])))


def test_unconstrained_rejects_short_outputs():
    import torch
    from paper_1512_01641_gb300 import miner
    batch = synth.make_batch(703, 3, v_src=500, v_tgt=500)
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    counts = plan.count()
    cap = int(miner.lib().mine_unconstrained_link_capacity(plan.handle))
    assert cap == int(batch.src.doc_sizes().sum())
    short = {"link_off": torch.empty(4, dtype=torch.int64, device="cuda"),
             "link_i": torch.empty(cap - 1, dtype=torch.int32, device="cuda"),
             "link_j": torch.empty(cap - 1, dtype=torch.int32, device="cuda"),
             "link_s": torch.empty(cap - 1, dtype=torch.float32, device="cuda"),
             "pair_score": torch.empty(3, dtype=torch.float32, device="cuda")}
    with pytest.raises(miner.MinerError):
        plan.align_unconstrained(miner.MineParams(), counts, out=short)


def test_unconstrained_long_targets_vs_oracle():
    """Targets of 256 sentences and more take the block-per-pair kernel
    (segments of a few columns per thread, block scans): same scores and
    links as the oracle, ties validated as above."""
    from paper_1512_01641_gb300 import miner
    ns = [20, 33, 5, 2]
    ms = [300, 257, 400, 256]
    dic = synth.make_dictionary(np.random.Generator(np.random.PCG64(704)), 800, 800)
    batch = synth.make_batch(705, len(ns), dic=dic, planted_frac=0.0, src_sizes=ns, tgt_sizes=ms)
    p = miner.MineParams(thr=-1.0)
    g = _gpu(batch, p)
    ref = oracle.mine(batch, p.w, p.b, p.gap, p.thr, want_sim=True)
    for k in range(batch.n_pairs):
        s = ref["sim"][k]
        score, links = unconstrained.align(s, p.gap)
        assert abs(g["score"][k] - score) <= H_REL * max(1.0, abs(score)), (k, g["score"][k], score)
        path = [(i, j) for i, j, _ in g["links"][k]]
        if path != links:
            choice = [None] * s.shape[0]
            for i, j in path:
                choice[i] = j
            assert unconstrained.path_score(s, p.gap, choice) >= score - TIE_TOL, (k, path, links)
