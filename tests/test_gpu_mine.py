"""GPU parity of the mining path (counts, similarity, alignment, threshold)
against the FP64 oracle, through the C ABI.  Tolerances: tests/gpu_parity.py."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1512_01641_gb300 import synth

from gpu_parity import S_TOL, check_alignment, check_counts, per_pair, run_gpu

pytestmark = pytest.mark.gpu

W = (4.0, 4.0, -2.0, 1.0)


def _params(thr=0.5, gap=0.3, b=-3.0):
    from paper_1512_01641_gb300 import miner
    return miner.MineParams(w=W, b=b, gap=gap, thr=thr)


def _edge_batch():
    # sizes around the 32-row strip and 32-column block edges, single rows and
    # columns, and very unequal documents
    ns = [1, 1, 40, 31, 32, 33, 63, 64, 65, 5, 130, 97]
    ms = [1, 50, 1, 33, 32, 31, 64, 65, 63, 130, 5, 96]
    return synth.make_batch(77, len(ns), v_src=3000, v_tgt=3000, planted_frac=0.0,
                            src_sizes=ns, tgt_sizes=ms)


def _mixed_batch():
    return synth.make_batch(78, 60, v_src=5000, v_tgt=5000, size_median=40, size_hi=200)


def _long_sentence_batch():
    # sentences of up to 255 tokens (several 32-lane chunks, 8 counter planes,
    # the largest hash table) with a small vocabulary, so that counts are high
    rng = np.random.default_rng(5)
    v = 400
    lists = [sorted(set(rng.integers(0, v, size=int(rng.integers(1, 4))).tolist())) for _ in range(v)]

    def sent(n):
        return sorted(rng.integers(0, v, size=n).tolist())
    src = [[sent(int(rng.integers(1, 256))) for _ in range(n)] for n in (3, 35, 7)]
    tgt = [[sent(int(rng.integers(1, 256))) for _ in range(m)] for m in (40, 4, 33)]
    # one pair where target sentences are full translations (counts = lengths)
    return synth.from_lists(src, tgt, lists, v_tgt=v)


def _dense_translation_batch():
    # every source id has 3 translations: strips carry ~1700 translations, so
    # the planner splits their row tables into row groups
    rng = np.random.Generator(np.random.PCG64(9))
    dic = synth.make_dictionary(rng, 3000, 3000, kmin=3, kmax=3)
    return synth.make_batch(79, 8, dic=dic, size_median=70, size_hi=160)


def _fanout_batch(kmin, kmax, seed):
    # every source id with kmin..kmax translations: fan-out 4 fills the tile
    # kernel's fixed-width records (row groups of 16 and 8 rows), fan-out 6 is
    # counted by the strip kernel instead
    rng = np.random.Generator(np.random.PCG64(seed))
    dic = synth.make_dictionary(rng, 2000, 2000, kmin=kmin, kmax=kmax)
    return synth.make_batch(seed + 1, 10, dic=dic, size_median=50, size_hi=140)


BATCHES = {"single_40x45": synth.single_pair, "edges": _edge_batch, "mixed": _mixed_batch,
           "long_sentences": _long_sentence_batch, "dense_translations": _dense_translation_batch,
           "fanout_4": lambda: _fanout_batch(4, 4, 81), "fanout_1_to_6": lambda: _fanout_batch(1, 6, 83)}


@pytest.fixture(scope="module", params=list(BATCHES))
def case(request):
    batch = BATCHES[request.param]()
    p_all = _params(thr=-1.0)
    p = _params()
    ref_all = oracle.mine(batch, p.w, p.b, p.gap, p_all.thr, want_counts=True, want_sim=True)
    ref = {"links": [[x for x in d if x[2] >= p.thr] for d in ref_all["diag"]]}
    gpu_all = run_gpu(batch, p_all, want_scores=True)
    gpu = run_gpu(batch, p, want_counts=False)
    return request.param, batch, p, ref_all, ref, gpu_all, gpu


def test_counts_bit_exact(case):
    name, batch, p, ref_all, ref, gpu_all, gpu = case
    check_counts(batch, gpu_all, ref_all)


def test_features_and_similarity(case):
    name, batch, p, ref_all, ref, gpu_all, gpu = case
    off = gpu_all["plan"].cell_offsets
    for k in range(batch.n_pairs):
        c = ref_all["counts"][k]
        N, M = c.shape[:2]
        if N * M == 0:
            continue
        ls = np.array([len(x) for x in batch.src.doc(k)])
        lt = np.array([len(x) for x in batch.tgt.doc(k)])
        feat = per_pair(gpu_all["feat"], off, k, (N, M, 4))
        s = per_pair(gpu_all["s"], off, k, (N, M))
        for i in range(0, N, max(1, N // 13)):
            for j in range(0, M, max(1, M // 11)):
                f64 = oracle.features(c[i, j, 0], c[i, j, 1], ls[i], lt[j])
                assert np.array_equal(feat[i, j], f64.astype(np.float32)), (k, i, j)
        assert np.abs(s - ref_all["sim"][k]).max() <= S_TOL


def test_alignment_and_threshold(case):
    name, batch, p, ref_all, ref, gpu_all, gpu = case
    ties = check_alignment(batch, p, gpu_all, ref_all, gpu, ref)
    # unplanted pairs repeat the same (counts, lengths) often, so mathematically
    # tied alignments are common; each was validated above
    assert ties <= max(2, batch.n_pairs // 3), f"{ties} near-tie pairs of {batch.n_pairs}"


def test_fused_equals_count_then_align(case):
    name, batch, p, ref_all, ref, gpu_all, gpu = case
    import torch
    plan = gpu["plan"]
    counts = plan.count()
    out = plan.align(p, counts)
    torch.cuda.synchronize()
    for key in ("link_off", "pair_score"):
        assert torch.equal(out[key][: plan.n_pairs + (key == "link_off")],
                           gpu["out"][key][: plan.n_pairs + (key == "link_off")]), key
    n = int(out["link_off"][-1])
    for key in ("link_i", "link_j", "link_s"):
        assert torch.equal(out[key][:n], gpu["out"][key][:n]), key


@pytest.mark.parametrize("shift", [2, 6, 14])
def test_align_from_counts_at_any_address(shift):
    """mine_align reads the counts wherever the caller put them: a copy at a
    2-byte-aligned (not 16-byte-aligned) address gives the same links and
    scores, with tiled and untiled pairs."""
    import torch
    from paper_1512_01641_gb300 import miner
    ns = [300, 97, 5, 64, 40]
    ms = [410, 33, 300, 97, 700]
    batch = synth.make_batch(83, len(ns), v_src=4000, v_tgt=4000, planted_frac=0.5, src_sizes=ns, tgt_sizes=ms)
    p = _params()
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        plan.set_option("tile_min_cells", 1 << 14)
        plan.set_option("tile_min_rows", 33)
        plan.set_option("tile_cols", 64)
        counts = plan.count()
        ref = plan.align(p, counts)
        torch.cuda.synchronize()
        ref = {k: v.clone() for k, v in ref.items()}
        raw = torch.zeros(counts.numel() + 64, dtype=torch.uint8, device="cuda")
        moved = raw[shift:shift + counts.numel()]
        moved.copy_(counts.reshape(-1))
        assert moved.data_ptr() % 16 == shift % 16
        got = plan.align(p, moved)
        plan.check()
        _outputs_equal(ref, got, batch.n_pairs)


def test_deterministic():
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _mixed_batch()
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        a = plan.mine(_params())
        b = plan.mine(_params())
        torch.cuda.synchronize()
        n = int(a["link_off"][-1])
        assert torch.equal(a["link_off"], b["link_off"])
        assert torch.equal(a["pair_score"], b["pair_score"])
        for key in ("link_i", "link_j", "link_s"):
            assert torch.equal(a[key][:n], b[key][:n])


def test_empty_documents_and_no_pairs():
    import torch
    from paper_1512_01641_gb300 import miner
    dic = [[0], [1, 2], [3]]
    src = [[], [[0, 1]], [[1], [2, 2]], []]
    tgt = [[[0]], [], [[1, 3], [2]], []]
    batch = synth.from_lists(src, tgt, dic, v_tgt=4)
    p = _params()
    r = run_gpu(batch, p)
    ref = oracle.mine(batch, p.w, p.b, p.gap, p.thr)
    for k in range(4):
        assert abs(r["score"][k] - ref["score"][k]) <= 1e-6
        assert [(i, j) for i, j, _ in r["links"][k]] == [(i, j) for i, j, _ in ref["links"][k]]
    empty = synth.from_lists([], [], dic, v_tgt=4)
    with miner.Plan(miner.DeviceBatch.from_batch(empty)) as plan:
        out = plan.mine(p)
        torch.cuda.synchronize()
        assert int(out["link_off"][0]) == 0


def test_rejects_malformed_inputs():
    import torch
    from paper_1512_01641_gb300 import miner
    good = synth.make_batch(3, 2, v_src=100, v_tgt=100, size_median=6)

    def attempt(mut):
        b = synth.make_batch(3, 2, v_src=100, v_tgt=100, size_median=6)
        mut(b)
        with pytest.raises(miner.MinerError) as e:
            miner.Plan(miner.DeviceBatch.from_batch(b))
        assert e.value.code == miner.MINE_EINVAL

    def unsorted(b):
        b.src.tok[0], b.src.tok[1] = 99, 0  # sentences hold >= 5 tokens
    attempt(unsorted)

    def bad_id(b):
        b.tgt.tok[-1] = 100
    attempt(bad_id)

    def empty_sentence(b):
        b.src.sent_tok_off[1] = 0
    attempt(empty_sentence)

    def bad_dict(b):
        b.dic.tgt[0] = 1000
    attempt(bad_dict)
    # the good batch still plans
    with miner.Plan(miner.DeviceBatch.from_batch(good)):
        pass


@pytest.mark.slow
def test_wikipedia_batch_sampled_pairs():
    """10,000 Wikipedia-shaped pairs in one launch; 150 sampled pairs (the largest
    included) compared in full with the oracle."""
    batch = synth.wiki_batch()
    p_all = _params(thr=-1.0)
    gpu = run_gpu(batch, p_all, want_counts=True)
    sizes = batch.src.doc_sizes() * batch.tgt.doc_sizes()
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([np.argsort(sizes)[-3:], rng.choice(batch.n_pairs, 147, replace=False)]))
    sub = batch.subset(pick)
    ref = oracle.mine(sub, p_all.w, p_all.b, p_all.gap, p_all.thr, want_counts=True, want_sim=True)
    off = gpu["plan"].cell_offsets
    sel = {"counts": None, "score": gpu["score"][pick], "links": [gpu["links"][k] for k in pick]}
    for n, k in enumerate(pick):
        got = per_pair(gpu["counts"], off, k, ref["counts"][n].shape)
        assert np.array_equal(got, ref["counts"][n]), k
    ties = check_alignment(sub, p_all, sel, ref)
    assert ties <= len(pick) // 3


@pytest.mark.slow
def test_long_pair_5000x5000():
    """One 5000 x 5000 pair (the long pairs of the uneven batch): full oracle
    comparison of the pair score and path, sampled cell counts."""
    batch = synth.uneven_batch(n_pairs=0, n_long=1)
    p_all = _params(thr=-1.0)
    gpu = run_gpu(batch, p_all, want_counts=True)
    ref = oracle.mine(batch, p_all.w, p_all.b, p_all.gap, p_all.thr, want_sim=True)
    c = gpu["counts"].reshape(5000, 5000, 2)
    rng = np.random.default_rng(1)
    src, tgt = batch.src.doc(0), batch.tgt.doc(0)
    for i, j in rng.integers(0, 5000, size=(400, 2)):
        assert tuple(c[i, j]) == oracle.counts(src[i], tgt[j], batch.dic)
    sel = {"score": gpu["score"], "links": gpu["links"]}
    assert check_alignment(batch, p_all, sel, ref) <= 1


def _outputs_equal(a, b, n_pairs):
    import torch
    n = int(a["link_off"][-1])
    assert torch.equal(a["link_off"][: n_pairs + 1], b["link_off"][: n_pairs + 1])
    assert torch.equal(a["pair_score"][:n_pairs], b["pair_score"][:n_pairs])
    for key in ("link_i", "link_j", "link_s"):
        assert torch.equal(a[key][:n], b[key][:n]), key


@pytest.mark.parametrize("tile_cols", [32, 96, 128, 256])
def test_tiled_fill_equals_single_warp_fill(tile_cols):
    """The cooperative tiled fill (tile waits, boundary rows/columns) gives
    bit-identical results to one warp per pair, for tile widths that do and do
    not divide the pair widths."""
    import torch
    from paper_1512_01641_gb300 import miner
    ns = [300, 97, 64, 257, 40]
    ms = [410, 300, 97, 64, 700]
    batch = synth.make_batch(81, len(ns), v_src=4000, v_tgt=4000, planted_frac=0.0, src_sizes=ns, tgt_sizes=ms)
    p = _params(thr=-1.0)
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        plan.set_option("tile_min_cells", 1 << 40)  # one warp per pair
        ref = plan.mine(p)
        torch.cuda.synchronize()
        ref = {k: v.clone() for k, v in ref.items()}
        plan.set_option("tile_min_cells", 1)
        plan.set_option("tile_min_rows", 33)
        plan.set_option("tile_cols", tile_cols)
        got = plan.mine(p)
        plan.check()
        _outputs_equal(ref, got, batch.n_pairs)
    ora = oracle.mine(batch, p.w, p.b, p.gap, p.thr, want_sim=True)
    sel = {"score": got["pair_score"].cpu().numpy(), "links": miner.links_per_pair(got, batch.n_pairs)}
    check_alignment(batch, p, sel, ora)


def test_options_at_creation_equal_options_set_later():
    """A plan created with its tiling options (mine_plan_create_with_options)
    reports them and mines exactly what a plan whose options were set after
    creation (work lists rebuilt, while earlier work of the plan is in flight)
    mines."""
    import torch
    from paper_1512_01641_gb300 import miner
    ns = [300, 97, 64, 257, 40]
    ms = [410, 300, 97, 64, 700]
    batch = synth.make_batch(82, len(ns), v_src=4000, v_tgt=4000, src_sizes=ns, tgt_sizes=ms)
    p = _params()
    opts = {"tile_cols": 64, "tile_min_cells": 1, "tile_min_rows": 33}
    db = miner.DeviceBatch.from_batch(batch)
    with miner.Plan(db, options=opts) as plan:
        assert {k: plan.get_option(k) for k in opts} == opts
        assert plan.get_option("n_tile_flags") > 0
        a = plan.mine(p)
        plan.check()
        torch.cuda.synchronize()
        a = {k: v.clone() for k, v in a.items()}
    with miner.Plan(db) as plan:
        plan.mine(p)  # in flight while the options below rebuild the work lists
        for k, v in opts.items():
            plan.set_option(k, v)
        b = plan.mine(p)
        plan.check()
        _outputs_equal(a, b, batch.n_pairs)


def test_link_recount_by_warp_vote_matches_cached_counts():
    """Recounting the overlaps of the aligned pairs by warp vote gives exactly
    the similarities computed from the cached bit-sliced counts."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _mixed_batch()
    p = _params(thr=-1.0)
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        a = plan.mine(p)
        torch.cuda.synchronize()
        a = {k: v.clone() for k, v in a.items()}
        plan.set_option("link_recount", 1)
        b = plan.mine(p)
        plan.check()
        _outputs_equal(a, b, batch.n_pairs)


def test_graph_replay_equals_direct_launches():
    """mine_pairs as one captured CUDA graph gives the results of direct
    launches; new parameters or new output buffers re-capture it."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = _edge_batch()
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        plan.set_option("use_graph", 0)
        direct = {k: v.clone() for k, v in plan.mine(_params()).items()}
        direct2 = {k: v.clone() for k, v in plan.mine(_params(gap=0.2, thr=0.4)).items()}
        torch.cuda.synchronize()
        plan.set_option("use_graph", 1)
        out = plan.new_output()
        for _ in range(3):
            g = plan.mine(_params(), out)
        torch.cuda.synchronize()
        assert plan.get_option("graph_captures") == 1
        _outputs_equal(direct, g, batch.n_pairs)
        g2 = plan.mine(_params(gap=0.2, thr=0.4), out)
        torch.cuda.synchronize()
        assert plan.get_option("graph_captures") == 2
        _outputs_equal(direct2, g2, batch.n_pairs)
        g3 = plan.mine(_params(gap=0.2, thr=0.4))  # new output buffers
        torch.cuda.synchronize()
        assert plan.get_option("graph_captures") == 3
        _outputs_equal(direct2, g3, batch.n_pairs)
        plan.check()


def test_bounded_tile_wait_reports_timeout_and_recovers():
    """A tile flag that nothing sets (fault injection): the waiting tiles give
    up after a short bounded spin, mine_plan_check reports MINE_ETIMEOUT, the
    context stays usable, and the next normal run is correct."""
    import torch
    from paper_1512_01641_gb300 import miner
    ns, ms = [300, 40], [410, 50]
    batch = synth.make_batch(83, 2, v_src=3000, v_tgt=3000, planted_frac=0.0, src_sizes=ns, tgt_sizes=ms)
    p = _params(thr=-1.0)
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        plan.set_option("tile_min_cells", 1)
        plan.set_option("tile_min_rows", 33)
        plan.set_option("tile_cols", 64)
        assert plan.get_option("n_tile_flags") > 0
        ref = {k: v.clone() for k, v in plan.mine(p).items()}
        plan.check()
        plan.set_option("wait_limit", 2000)  # ~0.4 ms per wait
        plan.set_option("fault_skip_flag", 0)
        plan.mine(p)
        with pytest.raises(miner.MinerError) as e:
            plan.check()
        assert e.value.code == miner.MINE_ETIMEOUT
        plan.set_option("fault_skip_flag", -1)
        plan.set_option("wait_limit", 1 << 24)
        got = plan.mine(p)
        plan.check()
        _outputs_equal(ref, got, batch.n_pairs)


def test_destroy_while_mining_in_flight_then_reuse_pool():
    """mine_plan_destroy returns at once; the scratch goes back to the pool only
    after the plan's work has finished, so a plan destroyed with its mining
    still in flight on a side stream leaves that output intact, and a new plan
    that reuses the memory right away mines correctly."""
    import torch
    from paper_1512_01641_gb300 import miner
    a = synth.make_batch(95, 60, v_src=3000, v_tgt=3000)
    b = synth.make_batch(96, 50, v_src=3000, v_tgt=3000)
    p = _params()
    refs = []
    for bt in (a, b):
        with miner.Plan(miner.DeviceBatch.from_batch(bt)) as plan:
            out = plan.mine(p)
            torch.cuda.synchronize()
            refs.append({k: v.clone() for k, v in out.items()})
    side = torch.cuda.Stream()
    for rep in range(3):
        pa = miner.Plan(miner.DeviceBatch.from_batch(a), stream=side)
        with torch.cuda.stream(side):
            oa = pa.mine(p, stream=side)
        pa.close()  # work still in flight on `side`
        with miner.Plan(miner.DeviceBatch.from_batch(b)) as pb:
            ob = pb.mine(p)
            torch.cuda.synchronize()
            _outputs_equal(refs[1], ob, b.n_pairs)
        side.synchronize()
        _outputs_equal(refs[0], oa, a.n_pairs)


@pytest.mark.slow
def test_uneven_batch_full_size_in_the_bench_launch_configuration():
    """The bench workload as the bench launches it: 100,000 Wikipedia-shaped
    pairs + 8 pairs of 5,000 x 5,000 sentences in one graph-replayed
    mine_pairs with 64-column tiles.  200 sampled small pairs (the largest
    included) are compared in full with the oracle (counts, score, path), two
    long pairs by score and path, and every long pair on 400 sampled cells of
    its counts."""
    import torch
    from paper_1512_01641_gb300 import miner
    batch = synth.uneven_batch()
    n = batch.n_pairs
    p_all = _params(thr=-1.0)
    with miner.Plan(miner.DeviceBatch.from_batch(batch)) as plan:
        plan.set_option("tile_cols", 64)
        plan.set_option("tile_min_cells", 1 << 20)
        plan.mine(p_all)
        out = plan.mine(p_all)  # graph replay
        counts = plan.count()
        torch.cuda.synchronize()
        assert plan.get_option("graph_captures") >= 1
        plan.check()
        off = plan.cell_offsets
        score = out["pair_score"][:n].cpu().numpy()
        links = miner.links_per_pair(out, n)
        sizes = batch.src.doc_sizes() * batch.tgt.doc_sizes()
        rng = np.random.default_rng(5)
        small = np.arange(n - 8)
        pick = np.unique(np.concatenate([small[np.argsort(sizes[small])[-5:]], rng.choice(small, 195, replace=False)]))
        sub = batch.subset(pick)
        ref = oracle.mine(sub, p_all.w, p_all.b, p_all.gap, p_all.thr, want_counts=True, want_sim=True)
        for x, k in enumerate(pick):
            got = counts[off[k]:off[k + 1]].cpu().numpy().reshape(ref["counts"][x].shape)
            assert np.array_equal(got, ref["counts"][x]), k
        ties = check_alignment(sub, p_all, {"score": score[pick], "links": [links[k] for k in pick]}, ref)
        assert ties <= len(pick) // 3
        for k in (n - 8, n - 7):
            one = batch.subset(np.array([k]))
            r1 = oracle.mine(one, p_all.w, p_all.b, p_all.gap, p_all.thr, want_sim=True)
            assert check_alignment(one, p_all, {"score": score[[k]], "links": [links[k]]}, r1) <= 1
        for k in range(n - 8, n):
            src, tgt = batch.src.doc(k), batch.tgt.doc(k)
            c = counts[off[k]:off[k + 1]].view(5000, 5000, 2)
            for i, j in rng.integers(0, 5000, size=(400, 2)):
                assert tuple(c[i, j].tolist()) == oracle.counts(src[i], tgt[j], batch.dic), (k, i, j)
