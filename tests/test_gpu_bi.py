"""Bi-directional mining (Section 5.4, BI) on the GPU against the oracle:
the dictionary transpose (bit-exact), the reverse direction mined by a plan
over the reversed batch, and the per-pair union / intersection of the two
directions' links."""
import math

import numpy as np
import pytest

import oracle
from oracle import bi
from paper_1512_01641_gb300 import synth
from gpu_parity import S_TOL, check_alignment

pytestmark = pytest.mark.gpu


def _dev_dict(d):
    import torch
    return torch.from_numpy(d.off.astype(np.int32)).cuda(), torch.from_numpy(d.tgt.astype(np.int32)).cuda()


@pytest.mark.parametrize("case", ["uniform", "skewed"])
def test_dict_transpose_equals_oracle(case):
    from paper_1512_01641_gb300 import miner
    rng = np.random.Generator(np.random.PCG64(31))
    if case == "uniform":
        d = synth.make_dictionary(rng, 5000, 4000)
    else:
        # a few target ids shared by hundreds of sources (long reverse lists),
        # and many target ids that nothing translates to (empty lists)
        lists = [sorted(set(rng.choice(8, int(rng.integers(1, 4))).tolist()) |
                        ({int(rng.integers(100, 3000))} if rng.random() < 0.3 else set())) for _ in range(2000)]
        off = np.zeros(2001, np.int32)
        off[1:] = np.cumsum([len(x) for x in lists])
        d = synth.Dictionary(2000, 3000, off, np.array([t for x in lists for t in x], np.int32))
    ref = bi.transpose_dictionary(d)
    off, tgt = miner.dict_transpose(*_dev_dict(d), d.v_src, d.v_tgt)
    assert np.array_equal(off.cpu().numpy(), ref.off)
    assert np.array_equal(tgt.cpu().numpy(), ref.tgt)


@pytest.mark.parametrize("bad", ["id_out_of_range", "offsets_decrease", "offsets_end"])
def test_dict_transpose_rejects_malformed_dictionary(bad):
    from paper_1512_01641_gb300 import miner
    off = np.array([0, 2, 3, 5], np.int32)
    tgt = np.array([0, 4, 1, 2, 3], np.int32)
    if bad == "id_out_of_range":
        tgt[3] = 9
    elif bad == "offsets_decrease":
        off[2] = 1
    else:
        off[3] = 4
    o, t = _dev_dict(synth.Dictionary(3, 5, off, tgt))
    with pytest.raises(miner.MinerError):
        miner.dict_transpose(o, t, 3, 5)


def _mixed_bi_batch():
    rng = np.random.Generator(np.random.PCG64(77))
    dic = synth.make_dictionary(rng, 4000, 4000)
    return synth.make_batch(78, 40, dic=dic, size_median=40, size_hi=150)


P_FWD = dict(w=(4.0, 4.0, -2.0, 1.0), b=-3.0, gap=0.3, thr=0.5)
P_REV = dict(w=(3.5, 4.5, -2.0, 0.5), b=-2.8, gap=0.25, thr=0.45)


@pytest.mark.parametrize("mode", ["union", "intersect"])
def test_bidirectional_mining_equals_oracle(mode):
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _mixed_bi_batch()
    rbatch = bi.reversed_batch(batch)
    pf, pr = miner.MineParams(**P_FWD), miner.MineParams(**P_REV)
    db = miner.DeviceBatch.from_batch(batch)
    with miner.BiPlan(db) as plan:
        # thr = -1: whole paths of both directions, checked like any mining
        all_f, all_r, _ = plan.mine(miner.MineParams(**{**P_FWD, "thr": -1.0}),
                                    miner.MineParams(**{**P_REV, "thr": -1.0}), mode)
        gpu_all_f = {"score": all_f["pair_score"].cpu().numpy(), "links": miner.links_per_pair(all_f, batch.n_pairs)}
        gpu_all_r = {"score": all_r["pair_score"].cpu().numpy(), "links": miner.links_per_pair(all_r, batch.n_pairs)}
        of, orv, comb = plan.mine(pf, pr, mode)
        torch.cuda.synchronize()
        gf, gr = miner.links_per_pair(of, batch.n_pairs), miner.links_per_pair(orv, batch.n_pairs)
        coff = comb["link_off"].cpu().numpy()
        ci, cj = comb["link_i"].cpu().numpy(), comb["link_j"].cpu().numpy()
        csf, csr = comb["s_fwd"].cpu().numpy(), comb["s_rev"].cpu().numpy()
    ref_f_all = oracle.mine(batch, np.array(P_FWD["w"]), P_FWD["b"], P_FWD["gap"], -1.0, want_sim=True)
    ref_r_all = oracle.mine(rbatch, np.array(P_REV["w"]), P_REV["b"], P_REV["gap"], -1.0, want_sim=True)
    ties = check_alignment(batch, pf, gpu_all_f, ref_f_all)
    ties += check_alignment(rbatch, pr, gpu_all_r, ref_r_all)
    ref_f = oracle.mine(batch, np.array(P_FWD["w"]), P_FWD["b"], P_FWD["gap"], P_FWD["thr"])
    ref_r = oracle.mine(rbatch, np.array(P_REV["w"]), P_REV["b"], P_REV["gap"], P_REV["thr"])
    want = bi.combine(ref_f["links"], ref_r["links"], mode)
    exact = 0
    for k in range(batch.n_pairs):
        got = list(zip(ci[coff[k]:coff[k + 1]].tolist(), cj[coff[k]:coff[k + 1]].tolist()))
        # valid in any case: ascending (i, j), distinct, inside the pair
        assert got == sorted(set(got))
        N, M = batch.src.doc_sizes()[k], batch.tgt.doc_sizes()[k]
        assert all(0 <= i < N and 0 <= j < M for i, j in got)
        same_f = [(i, j) for i, j, _ in gf[k]] == [(i, j) for i, j, _ in ref_f["links"][k]]
        same_r = [(i, j) for i, j, _ in gr[k]] == [(i, j) for i, j, _ in ref_r["links"][k]]
        if not (same_f and same_r):
            continue  # a near-tie path or a near-threshold link in one direction (checked above)
        exact += 1
        assert got == [(i, j) for i, j, _, _ in want[k]], f"pair {k}"
        for x, (_, _, sf, sr) in enumerate(want[k]):
            a, b = csf[coff[k] + x], csr[coff[k] + x]
            assert (math.isnan(sf) and math.isnan(a)) or abs(a - sf) <= S_TOL, f"pair {k} s_fwd"
            assert (math.isnan(sr) and math.isnan(b)) or abs(b - sr) <= S_TOL, f"pair {k} s_rev"
    assert exact >= batch.n_pairs - max(2, ties + 2)


def test_bidirectional_union_finds_more_links_than_one_direction():
    # the point of BI (Table 3: more bi-sentences than MONO): the union keeps
    # every link of either direction, the intersection only those of both
    from paper_1512_01641_gb300 import miner
    batch = _mixed_bi_batch()
    with miner.BiPlan(miner.DeviceBatch.from_batch(batch)) as plan:
        of, orv, u = plan.mine(miner.MineParams(**P_FWD), miner.MineParams(**P_REV), "union")
        nu, nf, nr = int(u["link_off"][-1]), int(of["link_off"][-1]), int(orv["link_off"][-1])
        _, _, x = plan.mine(miner.MineParams(**P_FWD), miner.MineParams(**P_REV), "intersect")
        nx = int(x["link_off"][-1])
    assert nu == nf + nr - nx and nu >= max(nf, nr) and nx <= min(nf, nr)


def test_combine_rejects_plans_that_are_not_reverses():
    from paper_1512_01641_gb300 import miner
    batch = _mixed_bi_batch()
    db = miner.DeviceBatch.from_batch(batch)
    with miner.Plan(db) as a, miner.Plan(db) as b:
        oa, ob = a.mine(miner.MineParams()), b.mine(miner.MineParams())
        with pytest.raises(miner.MinerError):
            miner.combine_links(a, oa, b, ob)
