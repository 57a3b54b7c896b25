"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the FP64 oracle on the same seeded inputs.

Tolerances (written here, used by every parity test):
  counts            bit-exact (integers)
  features          bit-exact against the FP64 quotient rounded to FP32
  similarity s      |s_gpu - s_oracle| <= 2e-6  (FP32 sigmoid of an FP32 dot
                    product of four features: a few ulp of 1)
  pair score        |H_gpu - H_oracle| <= 1e-5 * max(1, |H_oracle|)
  aligned path      identical diagonal cells, except pairs whose GPU path
                    scores (re-scored by the oracle in FP64) within 1e-4 of the
                    optimum: those are near-ties (several correct answers),
                    counted, and must still be valid monotone alignments
  threshold         identical kept links, except cells whose FP64 similarity
                    lies within 1e-6 of the threshold (the decision belongs to
                    FP rounding)
"""
from __future__ import annotations

import numpy as np

import oracle

S_TOL = 2e-6
H_REL = 1e-5
TIE_TOL = 1e-4
THR_BAND = 1e-6


def run_gpu(batch, params, want_counts=True, want_scores=False):
    import torch
    from paper_1512_01641_gb300 import miner
    plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
    res = {"plan": plan}
    counts = plan.count()
    if want_counts:
        res["counts"] = counts.cpu().numpy()
    if want_scores:
        s, f = plan.score(params, counts, want_features=True)
        res["s"], res["feat"] = s.cpu().numpy(), f.cpu().numpy()
    out = plan.mine(params)
    torch.cuda.synchronize()
    res["out"] = out
    res["score"] = out["pair_score"].cpu().numpy()[:batch.n_pairs]
    res["links"] = miner.links_per_pair(out, batch.n_pairs)
    return res


def per_pair(arr, off, k, shape):
    return arr[off[k]:off[k + 1]].reshape(shape)


def check_counts(batch, gpu, ref):
    off = gpu["plan"].cell_offsets
    for k in range(batch.n_pairs):
        got = per_pair(gpu["counts"], off, k, ref["counts"][k].shape)
        if not np.array_equal(got, ref["counts"][k]):
            bad = np.argwhere(got != ref["counts"][k])[:5]
            raise AssertionError(f"pair {k}: counts differ at {bad.tolist()}")


def check_alignment(batch, params, gpu_all, ref, gpu_thr=None, ref_thr=None):
    """gpu_all / ref: runs with thr = -1 (every diagonal step kept) -> whole
    paths; gpu_thr / ref_thr: the same with the real threshold.  Returns the
    number of near-tie pairs."""
    ties = 0
    for k in range(batch.n_pairs):
        h = ref["score"][k]
        g = float(gpu_all["score"][k])
        assert abs(g - h) <= H_REL * max(1.0, abs(h)), f"pair {k}: score {g} vs {h}"
        gd = [(i, j) for i, j, _ in gpu_all["links"][k]]
        od = [(i, j) for i, j, _ in ref["diag"][k]]
        S = ref["sim"][k]
        # link similarities agree with the oracle's
        for i, j, s in gpu_all["links"][k]:
            assert abs(s - S[i, j]) <= S_TOL, f"pair {k}: link ({i},{j}) s {s} vs {S[i, j]}"
        if gd != od:
            v = oracle.path_score(S, params.gap, gd)  # raises if not monotone
            assert v >= h - TIE_TOL, f"pair {k}: GPU path scores {v}, optimum {h} (not a near-tie)"
            ties += 1
            continue
        if gpu_thr is not None:
            gl = {(i, j) for i, j, _ in gpu_thr["links"][k]}
            ol = {(i, j) for i, j, _ in ref_thr["links"][k]}
            for (i, j) in gl ^ ol:
                assert abs(S[i, j] - params.thr) <= THR_BAND, f"pair {k}: link ({i},{j}) s={S[i, j]} thr"
            assert all(s >= params.thr for _, _, s in gpu_thr["links"][k])
            # ascending order
            lk = [(i, j) for i, j, _ in gpu_thr["links"][k]]
            assert lk == sorted(lk)
    return ties
