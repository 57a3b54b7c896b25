"""Streaming batches from host memory through BatchPipeline gives, batch by
batch, exactly the links and scores of Plan.mine on the same batch (with the
pipeline's plans at the default options, and with every pair of a batch
filled as tiles: the fill's arithmetic per cell does not depend on tiling)."""
import numpy as np
import pytest

from paper_1512_01641_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("options", [None, {"tile_cols": 64, "tile_min_cells": 1 << 12, "tile_min_rows": 32}],
                         ids=["default", "tiled"])
def test_pipeline_results_equal_plan_mine(options):
    import torch
    from paper_1512_01641_gb300 import miner
    from paper_1512_01641_gb300.pipeline import BatchPipeline
    rng = np.random.Generator(np.random.PCG64(11))
    dic = synth.make_dictionary(rng, 3000, 3000)
    batches = [synth.make_batch(90 + k, 40 + 7 * k, dic=dic) for k in range(4)]
    params = miner.MineParams()
    ref = []
    for b in batches:
        with miner.Plan(miner.DeviceBatch.from_batch(b)) as plan:
            out = plan.mine(params)
            n = int(out["link_off"][-1])
            ref.append({"link_off": out["link_off"].cpu(), "pair_score": out["pair_score"][:plan.n_pairs].cpu(),
                        "link_i": out["link_i"][:n].cpu(), "link_j": out["link_j"][:n].cpu(),
                        "link_s": out["link_s"][:n].cpu()})
    pipe = BatchPipeline(params, dic.v_src, dic.v_tgt, options=options)
    got = []
    for b in batches:
        host = [b.src.doc_sent_off, b.src.sent_tok_off, b.src.tok, b.tgt.doc_sent_off, b.tgt.sent_tok_off,
                b.tgt.tok, b.dic.off, b.dic.tgt]
        r = pipe.submit([torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in host])
        if r is not None:
            got.append(r)
    got.append(pipe.flush())
    assert pipe.flush() is None
    assert len(got) == len(batches)
    for a, b in zip(ref, got):
        for k in a:
            assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_buffer_entry_point_equals_plan_mine(pinned):
    """mine_pairs_host (inputs and outputs in host memory, one C-ABI call)
    gives exactly the links and scores of Plan.mine on device buffers; a
    short output is rejected."""
    import torch
    from paper_1512_01641_gb300 import miner
    b = synth.make_batch(97, 60, v_src=3000, v_tgt=3000)
    params = miner.MineParams()
    with miner.Plan(miner.DeviceBatch.from_batch(b)) as plan:
        out = plan.mine(params)
        n = int(out["link_off"][-1])
        ref = {"link_off": out["link_off"].cpu(), "pair_score": out["pair_score"][:plan.n_pairs].cpu(),
               "link_i": out["link_i"][:n].cpu(), "link_j": out["link_j"][:n].cpu(), "link_s": out["link_s"][:n].cpu()}
        cap = plan.link_capacity
    host = [b.src.doc_sent_off, b.src.sent_tok_off, b.src.tok, b.tgt.doc_sent_off, b.tgt.sent_tok_off, b.tgt.tok,
            b.dic.off, b.dic.tgt]
    host = [torch.from_numpy(np.ascontiguousarray(a)) for a in host]
    if pinned:
        host = [t.pin_memory() for t in host]
    got = miner.mine_host(host, b.dic.v_src, b.dic.v_tgt, params)
    m = int(got["link_off"][-1])
    assert m == n
    assert torch.equal(got["link_off"], ref["link_off"])
    assert torch.equal(got["pair_score"][:b.n_pairs], ref["pair_score"])
    for k in ("link_i", "link_j", "link_s"):
        assert torch.equal(got[k][:m], ref[k]), k
    short = {k: v.clone() for k, v in got.items()}
    for k in ("link_i", "link_j", "link_s"):
        short[k] = short[k][:cap - 1].clone()
    with pytest.raises(miner.MinerError):
        miner.mine_host(host, b.dic.v_src, b.dic.v_tgt, params, out=short)


@pytest.mark.parametrize("chunks", [2, 3, 7])
def test_host_entry_in_chunks_equals_plan_mine(chunks):
    """mine_pairs_host mining the batch as 2, 3 or 7 chunks of pairs (each
    with its own plan, the next chunk's upload and plan overlapping the
    current chunk's mining) gives exactly the links and scores of one plan
    over the batch; pairs of every size, empty documents included."""
    import torch
    from paper_1512_01641_gb300 import miner
    sizes = np.array([0, 3, 40, 1, 70, 5, 0, 33, 12, 90, 7, 2, 64, 31, 20, 9, 1, 45, 3, 0, 28])
    b = synth.make_batch(98, len(sizes), v_src=3000, v_tgt=3000, src_sizes=sizes)
    params = miner.MineParams()
    with miner.Plan(miner.DeviceBatch.from_batch(b)) as plan:
        out = plan.mine(params)
        n = int(out["link_off"][-1])
        ref = {"link_off": out["link_off"].cpu(), "pair_score": out["pair_score"][:plan.n_pairs].cpu(),
               "link_i": out["link_i"][:n].cpu(), "link_j": out["link_j"][:n].cpu(), "link_s": out["link_s"][:n].cpu()}
    host = [b.src.doc_sent_off, b.src.sent_tok_off, b.src.tok, b.tgt.doc_sent_off, b.tgt.sent_tok_off, b.tgt.tok,
            b.dic.off, b.dic.tgt]
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in host]
    got = miner.mine_host(host, b.dic.v_src, b.dic.v_tgt, params, options={"host_chunks": chunks})
    assert int(got["link_off"][-1]) == n
    assert torch.equal(got["link_off"], ref["link_off"])
    assert torch.equal(got["pair_score"][:b.n_pairs], ref["pair_score"])
    for k in ("link_i", "link_j", "link_s"):
        assert torch.equal(got[k][:n], ref[k]), k
