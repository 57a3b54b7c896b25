"""The allocation-free single-pair entry point (mine_align_pair_noalloc).

It exists for callers that cannot allocate device memory when they call (a
serving loop with a fixed memory budget, a library inside a framework that
owns every device allocation, code that cannot take cudaMalloc's implicit
synchronisation); its scratch is a fixed array inside the library.  Checked
here against the plan-based mine_align on the same counts, on two calls in a
row, through the C ABI.  This file is collected last so that a run stopping
at the first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1512_01641_gb300 import miner, synth

pytestmark = pytest.mark.gpu

MAX_SIDE = 2048
H_REL = 1e-5  # the pair-score tolerance of the parity tests


def _call(L, sent_s, sent_t, n, m, counts, params, out, stream):
    p = params.c()
    return L.mine_align_pair_noalloc(C.c_void_p(sent_s), C.c_void_p(sent_t), n, m, C.c_void_p(counts),
                                     C.byref(p), C.c_void_p(out["i"].data_ptr()), C.c_void_p(out["j"].data_ptr()),
                                     C.c_void_p(out["s"].data_ptr()), C.c_void_p(out["n"].data_ptr()),
                                     C.c_void_p(out["score"].data_ptr()), C.c_void_p(stream))


def test_noalloc_matches_plan_alignment_twice():
    import torch
    L = miner.lib(build_if_missing=True)
    ns = [40, 1, 130, 300, 77, 0, 5]
    ms = [45, 9, 97, 280, 1, 12, 0]
    batch = synth.make_batch(91, len(ns), v_src=4000, v_tgt=4000, planted_frac=0.0, src_sizes=ns, tgt_sizes=ms)
    params = miner.MineParams()
    db = miner.DeviceBatch.from_batch(batch)
    with miner.Plan(db) as plan:
        counts = plan.count()
        ref = plan.align(params, counts)
        torch.cuda.synchronize()
        ref_links = miner.links_per_pair(ref, batch.n_pairs)
        ref_score = ref["pair_score"].cpu().numpy()
        sent_s, sent_t = db.src[1], db.tgt[1]
        doc_s, doc_t = batch.src.doc_sent_off, batch.tgt.doc_sent_off
        stream = torch.cuda.current_stream().cuda_stream
        for rep in range(2):
            for k in range(batch.n_pairs):
                n, m = ns[k], ms[k]
                cap = max(min(n, m), 1)
                out = {"i": torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
                       "j": torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
                       "s": torch.full((cap,), -7.0, dtype=torch.float32, device="cuda"),
                       "n": torch.full((1,), -7, dtype=torch.int32, device="cuda"),
                       "score": torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")}
                cptr = counts.data_ptr() + 2 * int(plan.cell_offsets[k])
                rc = _call(L, sent_s.data_ptr() + 8 * int(doc_s[k]), sent_t.data_ptr() + 8 * int(doc_t[k]),
                           n, m, cptr, params, out, stream)
                assert rc == miner.MINE_OK, (rep, k, rc)
                torch.cuda.synchronize()
                nl = int(out["n"].item())
                got = list(zip(out["i"][:nl].tolist(), out["j"][:nl].tolist(), out["s"][:nl].tolist()))
                assert [(i, j) for i, j, _ in got] == [(i, j) for i, j, _ in ref_links[k]], (rep, k)
                assert np.allclose([s for *_, s in got], [s for *_, s in ref_links[k]], rtol=0, atol=2e-6)
                h = float(ref_score[k])
                assert abs(float(out["score"].item()) - h) <= H_REL * max(1.0, abs(h)), (rep, k)


def test_noalloc_rejects_oversized_pairs():
    L = miner.lib(build_if_missing=True)
    params = miner.MineParams()
    p = params.c()
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    for n, m in [(MAX_SIDE + 1, 10), (10, MAX_SIDE + 1), (-1, 3)]:
        rc = L.mine_align_pair_noalloc(dummy, dummy, n, m, dummy, C.byref(p), dummy, dummy, dummy, dummy, dummy,
                                       None)
        assert rc == miner.MINE_EINVAL
