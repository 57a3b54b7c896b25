"""Streaming mining of batches that live in host memory.

A serving loop receives one batch of document pairs after another in
(pinned) host memory.  ``BatchPipeline`` keeps the work stream busy with
mining: while batch b is mined, batch b+1's arrays are uploaded and its plan
is created (validation kernels, geometry, work lists; ``mine_plan_create``
waits only on its own stream) on a copy stream, and batch b+1's mining is
enqueued behind batch b's before batch b's links and scores are read back on a
third stream.  Streams and events only: every step of the path runs in the
library's kernels.
"""
from __future__ import annotations

from . import miner

HOST_ARRAYS = ("src.doc_sent_off", "src.sent_tok_off", "src.tok", "tgt.doc_sent_off", "tgt.sent_tok_off",
               "tgt.tok", "dict.off", "dict.tgt")


class BatchPipeline:
    """submit(host arrays) -> the previous batch's results (or None);
    flush() -> the last batch's results.

    host arrays: the eight CPU tensors of HOST_ARRAYS (pinned for overlap),
    in that order.  options: plan options (miner.OPTIONS names, e.g. the fill
    tile settings an autotuner chose) set on every batch's plan.  Results:
    dict of CPU tensors link_off, pair_score, link_i, link_j, link_s (the kept
    links of every pair, see mine_pairs)."""

    def __init__(self, params: miner.MineParams, v_src: int, v_tgt: int, options: dict | None = None):
        import torch
        self.params = params
        self.v_src, self.v_tgt = v_src, v_tgt
        self.options = dict(options or {})
        self.copy = torch.cuda.Stream()
        self.work = torch.cuda.Stream()
        self.down = torch.cuda.Stream()
        self._inflight = None

    def submit(self, host):
        import torch
        with torch.cuda.stream(self.copy):
            dev = [t.to("cuda", non_blocking=True) for t in host]
        for t in dev:
            t.record_stream(self.work)  # used by the mining on the work stream
        plan = miner.Plan(miner.DeviceBatch(*dev, self.v_src, self.v_tgt), stream=self.copy, options=self.options)
        ready = torch.cuda.Event()
        ready.record(self.copy)
        self.work.wait_event(ready)
        with torch.cuda.stream(self.work):
            out = plan.mine(self.params, stream=self.work)
        done = torch.cuda.Event()
        done.record(self.work)
        prev = self._collect()  # runs while this batch's mining waits behind the previous one
        self._inflight = (plan, dev, out, done)
        return prev

    def flush(self):
        prev = self._collect()
        self._inflight = None
        return prev

    def _collect(self):
        if self._inflight is None:
            return None
        import torch
        plan, dev, out, done = self._inflight
        self.down.wait_event(done)
        with torch.cuda.stream(self.down):
            off = out["link_off"].cpu()  # waits for this batch's mining
            n = int(off[-1])
            res = {"link_off": off, "pair_score": out["pair_score"][:plan.n_pairs].cpu(),
                   "link_i": out["link_i"][:n].cpu(), "link_j": out["link_j"][:n].cpu(),
                   "link_s": out["link_s"][:n].cpu()}
        plan.close()
        self._inflight = None
        return res
