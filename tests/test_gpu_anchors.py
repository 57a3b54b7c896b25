"""Anchor tokens (Section 5.3) on the GPU against the oracle: the extended
corpora and dictionary (bit-exact), mining of the extended batch (counts
bit-exact, alignments as every parity test checks them), and the effect the
section describes -- shared anchors mark parallel sentences."""
import numpy as np
import pytest

import oracle
from oracle import anchors as oracle_anchors
from paper_1512_01641_gb300 import synth
from gpu_parity import check_alignment, per_pair

pytestmark = pytest.mark.gpu

V_ANCHOR = 5000


def _dev_anchors(a):
    import torch
    return torch.from_numpy(a.sent_off.astype(np.int64)).cuda(), torch.from_numpy(a.ids.astype(np.int32)).cuda()


def _batch_and_anchors(seed=320, n=30, p_keep=0.9):
    rng = np.random.Generator(np.random.PCG64(seed))
    dic = synth.make_dictionary(rng, 4000, 4000)
    b = synth.make_batch(seed + 1, n, dic=dic, size_median=30, size_hi=90)
    sa, ta = synth.make_anchors(b, seed + 2, v_anchor=V_ANCHOR, p_anchor=0.4, p_keep=p_keep)
    return b, sa, ta


def test_extended_batch_equals_oracle():
    from paper_1512_01641_gb300 import miner
    b, sa, ta = _batch_and_anchors()
    e = oracle_anchors.extend_batch(b, sa, ta, V_ANCHOR)
    g = miner.add_anchors(miner.DeviceBatch.from_batch(b), _dev_anchors(sa), _dev_anchors(ta), V_ANCHOR)
    for got, want in ((g.src, e.src), (g.tgt, e.tgt)):
        assert np.array_equal(got[0].cpu().numpy(), want.doc_sent_off)
        assert np.array_equal(got[1].cpu().numpy(), want.sent_tok_off)
        assert np.array_equal(got[2].cpu().numpy(), want.tok)
    assert (g.v_src, g.v_tgt) == (e.dic.v_src, e.dic.v_tgt)
    assert np.array_equal(g.dict_off.cpu().numpy(), e.dic.off)
    assert np.array_equal(g.dict_tgt.cpu().numpy(), e.dic.tgt)


def test_mining_with_anchors_equals_oracle():
    import torch
    from paper_1512_01641_gb300 import miner
    b, sa, ta = _batch_and_anchors(330, 24)
    e = oracle_anchors.extend_batch(b, sa, ta, V_ANCHOR)
    g = miner.add_anchors(miner.DeviceBatch.from_batch(b), _dev_anchors(sa), _dev_anchors(ta), V_ANCHOR)
    p = miner.MineParams()
    p_all = miner.MineParams(thr=-1.0)
    ref = oracle.mine(e, np.array(p.w), p.b, p.gap, -1.0, want_counts=True, want_sim=True)
    with miner.Plan(g) as plan:
        counts = plan.count().cpu().numpy()
        off = plan.cell_offsets
        for k in range(b.n_pairs):
            assert np.array_equal(per_pair(counts, off, k, ref["counts"][k].shape), ref["counts"][k]), f"pair {k}"
        out = plan.mine(p_all)
        torch.cuda.synchronize()
        gpu = {"score": out["pair_score"].cpu().numpy(), "links": miner.links_per_pair(out, b.n_pairs)}
    ties = check_alignment(e, p, gpu, ref)
    assert ties <= max(2, b.n_pairs // 3), f"{ties} near-tie pairs of {b.n_pairs}"


def test_anchors_mark_parallel_sentences():
    # Section 5.3: sentences sharing names, dates, numbers or references are
    # likely translations -- with the anchors the default classifier keeps
    # more of the gold links of planted pairs at about the same precision
    from paper_1512_01641_gb300 import miner
    rng = np.random.Generator(np.random.PCG64(340))
    dic = synth.make_dictionary(rng, 4000, 4000)
    b = synth.make_batch(341, 200, dic=dic, planted_frac=1.0, p_wdrop=0.4, size_median=30, size_hi=90)
    sa, ta = synth.make_anchors(b, 342, v_anchor=V_ANCHOR, p_anchor=0.5, p_keep=0.9)
    db = miner.DeviceBatch.from_batch(b)
    gold = [set(map(tuple, g.tolist())) for g in b.gold]

    def score(batch):
        with miner.Plan(batch) as plan:
            links = miner.links_per_pair(plan.mine(miner.MineParams()), b.n_pairs)
        tp = sum(len({(i, j) for i, j, _ in l} & g) for l, g in zip(links, gold))
        return tp, sum(len(l) for l in links) - tp
    tp0, fp0 = score(db)
    tp1, fp1 = score(miner.add_anchors(db, _dev_anchors(sa), _dev_anchors(ta), V_ANCHOR))
    assert tp1 > tp0
    assert fp1 / max(tp1 + fp1, 1) <= fp0 / max(tp0 + fp0, 1) + 0.01


@pytest.mark.parametrize("bad", ["id_out_of_range", "offsets_end", "word_offsets_decrease"])
def test_add_anchors_rejects_malformed_anchor_lists(bad):
    # the checks run before anything is read through the offsets
    import torch
    from paper_1512_01641_gb300 import miner
    b, sa, ta = _batch_and_anchors(350, 4)
    ids = sa.ids.copy()
    off = sa.sent_off.copy()
    db = miner.DeviceBatch.from_batch(b)
    if bad == "id_out_of_range":
        ids[0] = V_ANCHOR
    elif bad == "offsets_end":
        off[-1] -= 1
    else:
        db.src[1][3] = db.src[1][2] - 1
    with pytest.raises(miner.MinerError):
        miner.add_anchors(db, (torch.from_numpy(off).cuda(), torch.from_numpy(ids).cuda()), _dev_anchors(ta), V_ANCHOR)


@pytest.mark.parametrize("bad", ["offsets_end", "offsets_decrease", "target_out_of_range"])
def test_dict_add_anchors_rejects_malformed_dictionaries(bad):
    # the dictionary is checked before its offsets are copied and shifted:
    # a malformed one is rejected with nothing written to the outputs
    import ctypes as C
    import torch
    from paper_1512_01641_gb300 import miner
    b, _, _ = _batch_and_anchors(351, 4)
    db = miner.DeviceBatch.from_batch(b)
    off = db.dict_off.clone()
    tgt = db.dict_tgt.clone()
    if bad == "offsets_end":
        off[-1] -= 1
    elif bad == "offsets_decrease":
        off[5] = off[4] - 1
    else:
        tgt[0] = db.v_tgt
    d = miner._Dict(db.v_src, db.v_tgt, tgt.numel(), off.data_ptr(), tgt.data_ptr())
    off_out = torch.full((db.v_src + V_ANCHOR + 1,), -5, dtype=torch.int32, device="cuda")
    tgt_out = torch.full((tgt.numel() + V_ANCHOR,), -5, dtype=torch.int32, device="cuda")
    rc = miner.lib().mine_dict_add_anchors(C.byref(d), V_ANCHOR, C.c_void_p(off_out.data_ptr()),
                                           C.c_void_p(tgt_out.data_ptr()), None)
    assert rc == miner.MINE_EINVAL
    torch.cuda.synchronize()
    assert bool((off_out == -5).all()) and bool((tgt_out == -5).all())
